// Measurement aids: the arithmetic ceiling of one selection
// (mmas_probe_draw_rate) and the L2 read bandwidth (mmas_probe_l2_bandwidth),
// both declared in include/mmas.h.
//
// A candidate-list step costs, per candidate slot, one Philox4x32-10 output
// word (a call yields four), the (0,1) uniform, its log2 (draw_log2), the key
// multiply by the reciprocal weight and a running maximum of the ordered key
// (Alg. 4 with log keys, Sec. 4.2.2).  This kernel runs exactly that work and
// nothing else -- no table loads, no tabu, no reductions -- at full occupancy,
// so its draw rate is the ALU ceiling the construction is measured against.
#include <algorithm>
#include <cstring>
#include <string>

#include "internal.cuh"
#include "mmas.h"

namespace mmas {
namespace {

__global__ void __launch_bounds__(256) k_draw_probe(ConstructArgs a, int iters, uint32_t *out)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    const float wi = 1.0f + (float)(threadIdx.x & 31) * 0.0625f;  // a reciprocal weight per slot
    uint32_t best = 0;
    for (int i = 0; i < iters; ++i) {
        uint4 r = make_uint4(threadIdx.x & 31, (uint32_t)i, g >> 5, 0x5EEDu);
        philox_rounds_rk<0, 10>(r, a.rk0, a.rk1);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t k = ord_key(__fmul_rn(draw_log2(unit_open(w[e])), wi));
            best = k > best ? k : best;
        }
    }
    out[g] = best;
}

// Read-only sweep of a buffer that stays resident in L2: every thread loads
// 16-byte words with a grid stride, `passes` times, through L2 only
// (ld.global.cg skips L1), and folds them into one word so no load is dead.
__global__ void __launch_bounds__(256) k_l2_probe(const uint4 *__restrict__ buf, size_t words, int passes,
                                                  uint32_t *out)
{
    const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    for (int p = 0; p < passes; ++p) {
#pragma unroll 4
        for (size_t i = g; i < words; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    out[g] = acc;
}

// Every draw value r = ((x >> 9) + 1/2) 2^-23 (x = k << 9, k = 0 .. 2^23 - 1):
// the largest relative error of draw_log2 and of the library's log2f against
// the double-precision log2.
__global__ void __launch_bounds__(256) k_draw_log2_error(unsigned long long *out)
{
    double e_draw = 0.0, e_lib = 0.0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < (1u << 23); k += gridDim.x * blockDim.x) {
        const float r = unit_open(k << 9);
        const double t = log2((double)r);  // r < 1: t < 0
        e_draw = fmax(e_draw, fabs((double)draw_log2(r) - t) / -t);
        e_lib = fmax(e_lib, fabs((double)log2f(r) - t) / -t);
    }
    // non-negative doubles: their bits order like their values
    atomicMax(out, (unsigned long long)__double_as_longlong(e_draw));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(e_lib));
}

}  // namespace
}  // namespace mmas

using namespace mmas;

extern "C" mmas_status mmas_debug_draw_log2_error(int32_t device, double *max_rel, double *max_rel_library)
{
    if (!max_rel) {
        set_thread_error("mmas_debug_draw_log2_error: max_rel must be non-NULL");
        return MMAS_EINVAL;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    unsigned long long *out = nullptr, h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(h));
    if (e == cudaSuccess) e = cudaMemset(out, 0, sizeof(h));
    if (e == cudaSuccess) {
        k_draw_log2_error<<<1024, 256>>>(out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
    if (out) cudaFree(out);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        set_thread_error(std::string("mmas_debug_draw_log2_error: ") + cudaGetErrorString(e));
        return MMAS_ECUDA;
    }
    double v[2];
    memcpy(v, h, sizeof(v));
    *max_rel = v[0];
    if (max_rel_library) *max_rel_library = v[1];
    return MMAS_OK;
}

extern "C" mmas_status mmas_probe_l2_bandwidth(int32_t device, int64_t bytes, double *gbs)
{
    if (!gbs || bytes < (1 << 20) || bytes > (int64_t)1 << 30) {
        set_thread_error("mmas_probe_l2_bandwidth: gbs must be non-NULL and 1 MiB <= bytes <= 1 GiB");
        return MMAS_EINVAL;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, device);
    uint4 *buf = nullptr;
    uint32_t *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 0.0;
    const size_t words = (size_t)bytes / sizeof(uint4);
    if (e == cudaSuccess) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_l2_probe, 256, 0);
        const int grid = prop.multiProcessorCount * (per_sm > 0 ? per_sm : 1);
        if (e == cudaSuccess) e = cudaMalloc(&buf, words * sizeof(uint4));
        if (e == cudaSuccess) e = cudaMemset(buf, 0x5A, words * sizeof(uint4));
        if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)grid * 256 * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        // about 1 ms a launch at tens of TB/s
        const int passes = (int)std::max<int64_t>(1, ((int64_t)32 << 30) / bytes);
        if (e == cudaSuccess) k_l2_probe<<<grid, 256>>>(buf, words, 1, out);  // bring it into L2
        for (int r = 0; e == cudaSuccess && r < 10; ++r) {
            cudaEventRecord(e0);
            k_l2_probe<<<grid, 256>>>(buf, words, passes, out);
            cudaEventRecord(e1);
            e = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && t > 0.0f)
                best = std::max(best, (double)words * sizeof(uint4) * passes / (t * 1e-3) / 1e9);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (out) cudaFree(out);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        set_thread_error(std::string("mmas_probe_l2_bandwidth: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MMAS_ENOMEM : MMAS_ECUDA;
    }
    *gbs = best;
    return MMAS_OK;
}

extern "C" mmas_status mmas_probe_draw_rate(int32_t device, float ms, double *draws_per_s)
{
    if (!draws_per_s || !(ms > 0.0f)) {
        set_thread_error("mmas_probe_draw_rate: draws_per_s must be non-NULL and ms > 0");
        return MMAS_EINVAL;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, device);
    uint32_t *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double rate = 0.0;
    if (e == cudaSuccess) {
        // full occupancy: as many 256-thread CTAs as fit, one wave
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_draw_probe, 256, 0);
        const int grid = prop.multiProcessorCount * (per_sm > 0 ? per_sm : 1);
        const size_t threads = (size_t)grid * 256;
        ConstructArgs a{};
        for (int r = 0; r < 10; ++r) {
            a.rk0[r] = 0x1234u + (uint32_t)r * 0x9E3779B9u;
            a.rk1[r] = 0x5678u + (uint32_t)r * 0xBB67AE85u;
        }
        if (e == cudaSuccess) e = cudaMalloc(&out, threads * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        int iters = 64;
        float t = 0.0f;
        // grow the launch until it runs for about `ms` (and at least 1 ms)
        for (int tries = 0; e == cudaSuccess && tries < 16; ++tries) {
            k_draw_probe<<<grid, 256>>>(a, iters, out);  // warm-up at this size
            cudaEventRecord(e0);
            k_draw_probe<<<grid, 256>>>(a, iters, out);
            cudaEventRecord(e1);
            e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e != cudaSuccess) break;
            rate = (double)threads * iters * 4.0 / (t * 1e-3);
            if (t >= ms || (t >= 1.0f && iters > (1 << 26))) break;
            const double scale = t > 0.0f ? ms / t : 64.0;
            iters = (int)std::min<double>((double)iters * (scale < 64.0 ? scale * 1.1 : 64.0), 1 << 28);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        set_thread_error(std::string("mmas_probe_draw_rate: ") + cudaGetErrorString(e));
        return MMAS_ECUDA;
    }
    *draws_per_s = rate;
    return MMAS_OK;
}
