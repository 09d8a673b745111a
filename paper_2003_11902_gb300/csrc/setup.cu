// Set-up kernels of a colony (Alg. 1 before the main loop; Sec. 2.1, Sec. 4.3):
// distances, heuristic weights, candidate lists, the nearest-neighbour tour,
// the initial trail limits and tau <- tau_max.  Run once per mmas_create.
#include <climits>

#include "distance.cuh"
#include "internal.cuh"

namespace mmas {

// d[i][j] = nint(|p_i - p_j|) for j < n; padding columns are left at zero.
// One thread per cell, rows striped over blockIdx.y.  Also tracks max(d).
__global__ void k_distances(const int2 *__restrict__ xy, int32_t n, int32_t ld,
                            int32_t *__restrict__ d, int *__restrict__ maxd)
{
    int local_max = 0;
    for (int i = blockIdx.y; i < n; i += gridDim.y) {
        const int2 pi = xy[i];
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
            const int32_t v = (i == j) ? 0 : euc2d_exact(pi, xy[j]);
            d[(size_t)i * ld + j] = v;
            local_max = max(local_max, v);
        }
    }
    local_max = __reduce_max_sync(0xFFFFFFFFu, (unsigned)local_max);
    if ((threadIdx.x & 31) == 0) atomicMax(maxd, local_max);
}

__global__ void k_max_dist(const int32_t *__restrict__ d, int32_t n, int32_t ld,
                           int *__restrict__ maxd)
{
    int local_max = 0;
    for (int i = blockIdx.y; i < n; i += gridDim.y)
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
            local_max = max(local_max, d[(size_t)i * ld + j]);
    local_max = __reduce_max_sync(0xFFFFFFFFu, (unsigned)local_max);
    if ((threadIdx.x & 31) == 0) atomicMax(maxd, local_max);
}

// eta_ij^beta with eta = 1/d (Sec. 2.1), d clamped to >= 1, zero diagonal,
// computed in double and rounded to float once.
__global__ void k_eta_beta(const int32_t *__restrict__ d, int32_t n, int32_t ld, double beta,
                           float *__restrict__ eb)
{
    for (int i = blockIdx.y; i < n; i += gridDim.y)
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
            float v = 0.0f;
            if (i != j) {
                const int32_t dij = d[(size_t)i * ld + j];
                const double dd = dij < 1 ? 1.0 : (double)dij;
                v = (float)pow(1.0 / dd, beta);
            }
            eb[(size_t)i * ld + j] = v;
        }
}

// The same values through a table: eta^beta depends on the integer distance
// only, so table[v] = pow(1 / max(v, 1), beta) for v = 0 .. maxd, computed once
// a distance value, is gathered for every cell (uniform n = 18,500: 14,143
// values for 342 M cells).
__global__ void k_eta_table(int32_t maxd, double beta, float *__restrict__ table)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= maxd; v += gridDim.x * blockDim.x) {
        const double dd = v < 1 ? 1.0 : (double)v;
        table[v] = (float)pow(1.0 / dd, beta);
    }
}

__global__ void k_eta_beta_table(const int32_t *__restrict__ d, int32_t n, int32_t ld,
                                 const float *__restrict__ table, float *__restrict__ eb)
{
    for (int i = blockIdx.y; i < n; i += gridDim.y)
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
            eb[(size_t)i * ld + j] = i != j ? __ldg(table + d[(size_t)i * ld + j]) : 0.0f;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Candidate lists (Sec. 4.3): the cl nearest other nodes of each row in
// ascending (distance, id) order, as 32-bit and/or 16-bit ids (either output
// may be null).  One warp per row, cl <= SELECT_MAX:
//  1. the cl-th smallest distance T of the row (j != i): the smallest T with at
//     least cl distances <= T, by bisection on [0, max] with one counting pass
//     of the row per halving (about log2 max passes);
//  2. the keys (d << 32 | j) of every node with d < T and of the lowest-id
//     nodes with d = T, cl in all, into the warp's shared memory (chunks of 32
//     consecutive ids in order, so the ties taken are the lowest ids);
//  3. a bitonic sort of those keys (padded to a power of two) in shared memory.
constexpr int SELECT_MAX = 1024;

__device__ __forceinline__ int pow2_at_least(int k)
{
    int p = 1;
    while (p < k) p <<= 1;
    return p;
}

__global__ void k_candidates(const int32_t *__restrict__ d, int32_t n, int32_t ld, int32_t cl,
                             int32_t *__restrict__ cand32, uint16_t *__restrict__ cand16)
{
    extern __shared__ unsigned long long s_keys[];  // pow2_at_least(cl) per warp
    const int lane = threadIdx.x & 31;
    const int kp = pow2_at_least(cl);
    unsigned long long *keys = s_keys + (size_t)(threadIdx.x >> 5) * kp;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const unsigned below = (1u << lane) - 1u;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int32_t *row = d + (size_t)i * ld;
        int mx = 0;
        for (int j = lane; j < n; j += 32)
            if (j != i) mx = row[j] > mx ? row[j] : mx;
        mx = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)mx);
        // 1. T: count(d <= lo) < cl <= count(d <= hi)
        long long lo = -1, hi = mx;
        int c_lo = 0;
        while (hi - lo > 1) {
            const int mid = (int)(lo + (hi - lo) / 2);
            int c = 0;
            for (int j = lane; j < n; j += 32) c += (j != i && row[j] <= mid) ? 1 : 0;
            c = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)c);
            if (c >= cl) {
                hi = mid;
            } else {
                lo = mid;
                c_lo = c;
            }
        }
        const int T = (int)hi;
        const int need_eq = cl - c_lo;  // nodes at distance T to take, lowest ids first
        // 2. collect
        int cnt = 0, eq = 0;
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            const int v = (j < n && j != i) ? row[j] : -1;
            const bool lt = v >= 0 && v < T;
            const bool te = v == T;
            const unsigned mte = __ballot_sync(0xFFFFFFFFu, te);
            const bool take = lt || (te && eq + __popc(mte & below) < need_eq);
            const unsigned mt = __ballot_sync(0xFFFFFFFFu, take);
            if (take) keys[cnt + __popc(mt & below)] = ((unsigned long long)(uint32_t)v << 32) | (uint32_t)j;
            cnt += __popc(mt);
            const int te_n = __popc(mte);
            eq += te_n < need_eq - eq ? te_n : need_eq - eq;
        }
        for (int e = cl + lane; e < kp; e += 32) keys[e] = ~0ull;
        __syncwarp();
        // 3. bitonic sort, ascending
        for (int size = 2; size <= kp; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = lane; t < (kp >> 1); t += 32) {
                    const int a = 2 * stride * (t / stride) + (t % stride), b = a + stride;
                    const unsigned long long ka = keys[a], kb = keys[b];
                    const bool up = (a & size) == 0;
                    if ((ka > kb) == up) {
                        keys[a] = kb;
                        keys[b] = ka;
                    }
                }
                __syncwarp();
            }
        }
        for (int e = lane; e < cl; e += 32) {
            const uint32_t j = (uint32_t)(keys[e] & 0xFFFFFFFFull);
            if (cand32) cand32[(size_t)i * cl + e] = (int32_t)j;
            if (cand16) cand16[(size_t)i * cl + e] = (uint16_t)j;
        }
        __syncwarp();  // the keys are read before the warp's next row writes them
    }
}

// Nearest-neighbour tour from node 0, ties -> lower id (one CTA, n sequential
// arg-min steps), and its length into sc->nn_len.  With a list of each row's
// nearest nodes in (distance, id) order (list: L entries a row, pitch P, 16-
// or 32-bit ids; L = 0: none), a step takes the first unvisited entry of the
// current row's list -- every node outside the list comes after all of its
// entries in that order -- and scans the row only when the whole list is
// visited.
template <typename T>
__global__ void __launch_bounds__(1024) k_nn_tour(const int32_t *__restrict__ d, int32_t n,
                                                  int32_t ld, int32_t *__restrict__ tour,
                                                  Scalars *sc, const T *__restrict__ list, int L, int P)
{
    extern __shared__ unsigned char vis[];
    __shared__ unsigned long long red[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int i = tid; i < n; i += blockDim.x) vis[i] = 0;
    __syncthreads();
    if (tid == 0) {
        vis[0] = 1;
        tour[0] = 0;
    }
    __syncthreads();
    int cur = 0;
    for (int t = 1; t < n; ++t) {
        unsigned long long b = ~0ull;
        if (L > 0) {  // the first unvisited entry of cur's list (the same in every thread)
            const T *lrow = list + (size_t)cur * P;
            unsigned long long e_best = ~0ull;
            for (int e = tid; e < L; e += blockDim.x) {
                const int v = (int)lrow[e];
                if (!vis[v]) {
                    const unsigned long long key = ((unsigned long long)(uint32_t)e << 32) | (uint32_t)v;
                    e_best = key < e_best ? key : e_best;
                }
            }
            e_best = warp_min_u64(e_best);
            if (lane == 0) red[warp] = e_best;
            __syncthreads();
            if (warp == 0) {
                unsigned long long v = lane < nwarps ? red[lane] : ~0ull;
                v = warp_min_u64(v);
                if (lane == 0) red[0] = v;
            }
            __syncthreads();
            b = red[0];
            __syncthreads();  // red is read before it is written again
        }
        if (b == ~0ull) {  // no list, or every listed node visited: scan the row
            const int32_t *row = d + (size_t)cur * ld;
            unsigned long long best = ~0ull;
            for (int j = tid; j < n; j += blockDim.x)
                if (!vis[j]) {
                    const unsigned long long key =
                        ((unsigned long long)(uint32_t)row[j] << 32) | (uint32_t)j;
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
            b = red[0];
        }
        const int nxt = (int)(b & 0xFFFFFFFFull);
        if (tid == 0) {
            vis[nxt] = 1;
            tour[t] = nxt;
        }
        cur = nxt;
        __syncthreads();
    }
    // the length, from the finished tour (written by thread 0, visible after
    // the barrier)
    long long part = 0;
    for (int t = tid; t < n; t += blockDim.x) {
        const int u = tour[t], v = tour[t + 1 < n ? t + 1 : 0];
        part += d[(size_t)u * ld + v];
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
    if (lane == 0) red[warp] = (unsigned long long)part;
    __syncthreads();
    if (tid == 0) {
        long long len = 0;
        for (int w = 0; w < nwarps; ++w) len += (long long)red[w];
        sc->nn_len = len;
    }
}

// Initial limits from the nearest-neighbour length, scalars reset, and
// tau <- tau_max on every real cell (padding columns stay zero).
__global__ void k_init_colony(int32_t n, int32_t ld, double rho, double p_root,
                              float *__restrict__ tau, Scalars *sc)
{
    __shared__ float s_tmax;
    if (threadIdx.x == 0) {
        float tx, tn;
        trail_limits(n, rho, p_root, sc->nn_len, &tx, &tn);
        s_tmax = tx;
        if (blockIdx.x == 0 && blockIdx.y == 0) {
            sc->tmax = tx;
            sc->tmin = tn;
        }
    }
    __syncthreads();
    const float tx = s_tmax;
    for (int i = blockIdx.y; i < n; i += gridDim.y)
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ld; j += gridDim.x * blockDim.x)
            tau[(size_t)i * ld + j] = j < n ? tx : 0.0f;
}

static dim3 cell_grid(int32_t n)
{
    const int gx = (n + 255) / 256;
    const int gy = n < 4096 ? n : 4096;
    return dim3(gx, gy);
}

cudaError_t launch_distances(const int2 *xy, int32_t n, int32_t ld, int32_t *d, int *maxd,
                             cudaStream_t s)
{
    k_distances<<<cell_grid(n), 256, 0, s>>>(xy, n, ld, d, maxd);
    return cudaGetLastError();
}

cudaError_t launch_max_dist(const int32_t *d, int32_t n, int32_t ld, int *maxd, cudaStream_t s)
{
    k_max_dist<<<cell_grid(n), 256, 0, s>>>(d, n, ld, maxd);
    return cudaGetLastError();
}

cudaError_t launch_eta_beta(const int32_t *d, int32_t n, int32_t ld, double beta, float *eb,
                            float *table, int32_t maxd, cudaStream_t s)
{
    if (table) {  // table: maxd + 1 floats (every distance lies in [0, maxd])
        k_eta_table<<<(maxd + 256) / 256 < 4096 ? (maxd + 256) / 256 : 4096, 256, 0, s>>>(maxd, beta, table);
        k_eta_beta_table<<<cell_grid(n), 256, 0, s>>>(d, n, ld, table, eb);
    } else {
        k_eta_beta<<<cell_grid(n), 256, 0, s>>>(d, n, ld, beta, eb);
    }
    return cudaGetLastError();
}

cudaError_t launch_candidates(const int32_t *d, int32_t n, int32_t ld, int32_t cl,
                              int32_t *cand32, uint16_t *cand16, cudaStream_t s)
{
    if (cl <= 0) return cudaSuccess;
    if (cl > SELECT_MAX) return cudaErrorInvalidValue;
    int kp = 1;
    while (kp < cl) kp <<= 1;
    const int threads = 128;  // 4 warps, one row each at a time
    const size_t smem = (size_t)(threads / 32) * kp * sizeof(unsigned long long);
    cudaError_t e = cudaFuncSetAttribute(k_candidates, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int rows_per_wave = 152 * 8 * (threads / 32);
    const int blocks = ((n < rows_per_wave ? n : rows_per_wave) * 32 + threads - 1) / threads;
    k_candidates<<<blocks, threads, smem, s>>>(d, n, ld, cl, cand32, cand16);
    return cudaGetLastError();
}

cudaError_t launch_nn_tour(const int32_t *d, int32_t n, int32_t ld, int32_t *tour, Scalars *sc,
                           const void *list, bool list16, int L, int P, cudaStream_t s)
{
    if (list16) {
        cudaError_t e = cudaFuncSetAttribute(k_nn_tour<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             65536);
        if (e != cudaSuccess) return e;
        k_nn_tour<uint16_t><<<1, 1024, (size_t)n, s>>>(d, n, ld, tour, sc, static_cast<const uint16_t *>(list),
                                                       L, P);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_nn_tour<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             65536);
        if (e != cudaSuccess) return e;
        k_nn_tour<int32_t><<<1, 1024, (size_t)n, s>>>(d, n, ld, tour, sc, static_cast<const int32_t *>(list),
                                                      list ? L : 0, P);
    }
    return cudaGetLastError();
}

cudaError_t launch_init_colony(int32_t n, int32_t ld, double rho, double p_root, float *tau,
                               Scalars *sc, cudaStream_t s)
{
    k_init_colony<<<dim3((ld + 255) / 256, n < 4096 ? n : 4096), 256, 0, s>>>(n, ld, rho, p_root,
                                                                              tau, sc);
    return cudaGetLastError();
}

}  // namespace mmas
