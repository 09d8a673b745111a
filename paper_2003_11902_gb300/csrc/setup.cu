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
// may be null).  One warp per row; cl rounds, each taking the smallest key
// (d << 32 | j) above the previous round's key.
__global__ void k_candidates(const int32_t *__restrict__ d, int32_t n, int32_t ld, int32_t cl,
                             int32_t *__restrict__ cand32, uint16_t *__restrict__ cand16)
{
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int32_t *row = d + (size_t)i * ld;
        unsigned long long last = 0;
        for (int r = 0; r < cl; ++r) {
            unsigned long long best = ~0ull;
            for (int j = lane; j < n; j += 32) {
                if (j == i) continue;
                const unsigned long long key =
                    ((unsigned long long)(uint32_t)row[j] << 32) | (uint32_t)j;
                if ((r == 0 || key > last) && key < best) best = key;
            }
            best = warp_min_u64(best);
            if (lane == 0) {
                if (cand32) cand32[(size_t)i * cl + r] = (int32_t)(best & 0xFFFFFFFFull);
                if (cand16) cand16[(size_t)i * cl + r] = (uint16_t)(best & 0xFFFFull);
            }
            last = best;
        }
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
                            cudaStream_t s)
{
    k_eta_beta<<<cell_grid(n), 256, 0, s>>>(d, n, ld, beta, eb);
    return cudaGetLastError();
}

cudaError_t launch_candidates(const int32_t *d, int32_t n, int32_t ld, int32_t cl,
                              int32_t *cand32, uint16_t *cand16, cudaStream_t s)
{
    if (cl <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (n * 32 + threads - 1) / threads;
    k_candidates<<<blocks, threads, 0, s>>>(d, n, ld, cl, cand32, cand16);
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
