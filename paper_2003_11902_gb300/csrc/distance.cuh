// Exact TSPLIB EUC_2D distance on the device, shared by the set-up, scoring,
// 2-opt and allocation-free kernels.
#pragma once

#include <cstdint>

namespace mmas {

// TSPLIB rounded Euclidean distance r = nint(sqrt(s)), s = dx^2 + dy^2, exact.
// r is the integer with r^2 - r < s <= r^2 + r (sqrt(s) is never a
// half-integer).
//
// Fast path, |dx|, |dy| < 2^17 (s < 2^35): the single-precision estimate
// s * rsqrt(s) has relative error under 2^-21, so it is within 0.1 of sqrt(s)
// and its rounding r0 is within 0.6 of sqrt(s): r0 is r or r +- 1.  Then
// e = s - r0^2 - r0 has |e| < 2^20, so it is exact in wrapping 32-bit
// arithmetic, and one comparison on each side settles r: r0 + 1 if e > 0,
// r0 - 1 if e + 2 r0 <= 0 (that is s <= r0^2 - r0, r0 > 0), else r0.
// Otherwise (points 2^17 or more apart on an axis) q = floor(sqrt(s)) comes
// from the double square root with 64-bit integer correction, and
// r = q + [s > q^2 + q].  |coords| < 2^30 keeps dx, dy in int32 and s < 2^63.
__device__ __forceinline__ int32_t euc2d_exact(int2 a, int2 b)
{
    const int32_t dx = a.x - b.x, dy = a.y - b.y;  // |coords| < 2^30: no overflow
    constexpr uint32_t H = (1u << 17) - 1u;  // |dx| <= H  <=>  dx + H in [0, 2H]
    if ((uint32_t)dx + H <= 2u * H && (uint32_t)dy + H <= 2u * H) {
        const float fx = (float)dx, fy = (float)dy;  // exact
        const float fs = __fmaf_rn(fx, fx, __fmul_rn(fy, fy));
        const float est = fs > 0.0f ? __fmul_rn(fs, rsqrtf(fs)) : 0.0f;
        const int32_t r0 = __float2int_rn(est);
        const uint32_t ud = (uint32_t)dx, ue = (uint32_t)dy, ur = (uint32_t)r0;
        const int32_t e = (int32_t)(ud * ud + ue * ue - ur * ur - ur);
        return r0 + (e > 0 ? 1 : 0) - ((r0 > 0 && e + 2 * r0 <= 0) ? 1 : 0);
    }
    const long long lx = dx, ly = dy;
    const unsigned long long s = (unsigned long long)(lx * lx) + (unsigned long long)(ly * ly);
    unsigned long long q = (unsigned long long)sqrt((double)s);
    while (q * q > s) --q;
    while ((q + 1) * (q + 1) <= s) ++q;
    return (int32_t)(q + (s > q * q + q ? 1ull : 0ull));
}

}  // namespace mmas
