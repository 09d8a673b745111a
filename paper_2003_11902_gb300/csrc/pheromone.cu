// The rest of an iteration after construction (Alg. 1; Sec. 2.1, Sec. 4.4):
//   k_best    iteration best (shortest tour, ties -> lower ant), global best
//             replaced by a strictly shorter tour, trail limits, the deposit
//             amount 1/C and each node's two neighbours in the deposited tour;
//   k_update  one streaming pass over the n x n matrices: evaporation with
//             both clamps, the deposit on the two tour edges of each row
//             (atomic-free: row i owns cells (i, succ(i)) and (i, pred(i)),
//             which covers both directions of every tour edge), then
//             choice_info = tau^alpha eta^beta, stored as-is (candidate-list
//             mode, for the fallback) or as its reciprocal (whole-row mode,
//             Sec. 4.2.2), plus 1/choice_info gathered for each candidate.
// The paper runs evaporation and deposition as two kernels (Sec. 4.4); here
// they are one pass, so each cell is read and written once per iteration.
#include <climits>

#include "internal.cuh"

namespace mmas {

namespace {

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

__global__ void __launch_bounds__(1024) k_best(const BestArgs a)
{
    __shared__ unsigned long long red[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    unsigned long long best = ~0ull;
    for (int k = tid; k < a.m; k += blockDim.x) {
        const unsigned long long key =
            ((unsigned long long)(uint32_t)a.lens[k] << 32) | (uint32_t)k;
        best = key < best ? key : best;
    }
    best = warp_min_u64(best);
    if (lane == 0) red[warp] = best;
    __syncthreads();
    if (warp == 0) {
        unsigned long long v = lane < nwarps ? red[lane] : ~0ull;
        v = warp_min_u64(v);
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    const unsigned long long b = red[0];
    const int ib = (int)(b & 0xFFFFFFFFull);
    const int len = (int)(b >> 32);
    Scalars *sc = a.sc;
    const int gb = sc->gb_len;
    const bool improved = len < gb;
    __syncthreads();  // every thread has read gb_len before it changes

    const int32_t *ibt = a.tours + (size_t)ib * a.ld;
    if (improved)
        for (int t = tid; t < a.n; t += blockDim.x) a.gb_tour[t] = ibt[t];
    if (tid == 0) {
        sc->ib_len = len;
        sc->ib_ant = ib;
        if (improved) {
            float tx, tn;
            trail_limits(a.n, a.rho, a.p_root, len, &tx, &tn);
            sc->gb_len = len;
            sc->tmax = tx;
            sc->tmin = tn;
        }
        const int dl = a.deposit ? (improved ? len : gb) : len;
        sc->dep_len = dl;
        sc->delta = (float)__ddiv_rn(1.0, (double)dl);
        if (a.advance) {
            sc->iter += 1;
            sc->iterations += 1;
        }
    }
    __syncthreads();  // the global-best copy is complete
    const int32_t *dep = a.deposit ? a.gb_tour : ibt;
    for (int t = tid; t < a.n; t += blockDim.x) {
        const int v = dep[t];
        const int nx = dep[t + 1 == a.n ? 0 : t + 1];
        const int pv = dep[t == 0 ? a.n - 1 : t - 1];
        a.nbr[v] = make_int2(nx, pv);
    }
}

template <bool FULLROW, bool ALPHA1>
__global__ void __launch_bounds__(256) k_update(const UpdateArgs a)
{
    const float tmin = a.sc->tmin, tmax = a.sc->tmax, delta = a.sc->delta;
    const int nq = a.ld >> 2;
    for (int i = blockIdx.x; i < a.n; i += gridDim.x) {
        int succ = -1, pred = -1;
        if (a.nbr) {
            const int2 nb = a.nbr[i];
            succ = nb.x;
            pred = nb.y;
        }
        float4 *trow = reinterpret_cast<float4 *>(a.tau + (size_t)i * a.ld);
        const float4 *erow = reinterpret_cast<const float4 *>(a.eb + (size_t)i * a.ld);
        float4 *wrow = reinterpret_cast<float4 *>(a.wmat + (size_t)i * a.ld);
#pragma unroll 2
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            const float4 t4 = trow[q];
            const float4 e4 = __ldg(erow + q);
            float tv[4] = {t4.x, t4.y, t4.z, t4.w};
            const float ev[4] = {e4.x, e4.y, e4.z, e4.w};
            float wv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = (q << 2) + c;
                float x = tv[c];
                if (j < a.n) {
                    if (a.evaporate) {
                        x = fminf(fmaxf(__fmul_rn(x, a.persist), tmin), tmax);
                        if (j == succ || j == pred) x = fminf(__fadd_rn(x, delta), tmax);
                    }
                    const float w = ALPHA1 ? __fmul_rn(x, ev[c]) : __fmul_rn(powf(x, a.alpha), ev[c]);
                    wv[c] = FULLROW ? __frcp_rn(w) : w;
                } else {
                    x = 0.0f;
                    wv[c] = 0.0f;
                }
                tv[c] = x;
            }
            trow[q] = make_float4(tv[0], tv[1], tv[2], tv[3]);
            wrow[q] = make_float4(wv[0], wv[1], wv[2], wv[3]);
        }
        if (!FULLROW && a.cl > 0) {
            __syncthreads();  // this row's choice_info is written and visible to the CTA
            const float *w1 = a.wmat + (size_t)i * a.ld;
            for (int c = threadIdx.x; c < a.cl; c += blockDim.x) {
                const int v = a.cand32[(size_t)i * a.cl + c];
                a.cwinv[(size_t)i * a.cl + c] = __frcp_rn(w1[v]);
            }
        }
    }
}

}  // namespace

cudaError_t launch_best(const BestArgs &a, cudaStream_t s)
{
    k_best<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_update(const UpdateArgs &a, int num_sms, cudaStream_t s)
{
    const int grid = a.n < num_sms * 8 ? a.n : num_sms * 8;
    const bool a1 = a.alpha == 1.0f;
    if (a.fullrow) {
        if (a1) k_update<true, true><<<grid, 256, 0, s>>>(a);
        else k_update<true, false><<<grid, 256, 0, s>>>(a);
    } else {
        if (a1) k_update<false, true><<<grid, 256, 0, s>>>(a);
        else k_update<false, false><<<grid, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace mmas
