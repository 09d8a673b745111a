// 2-opt local search (Sec. 5.7): Bentley's neighbour-list 2-opt with
// don't-look bits, first improvement, on whole tours.
//
// One CTA improves one tour held in shared memory (tour, position of each
// city, don't-look bits: 9 bytes per city).  The sequential search visits the
// cities in index order, skipping those whose don't-look bit is set; a city
// without a move gets its bit set, a move clears the bits of its four cities
// and the visit continues after the moving city; a run ends after a pass with
// no move, and runs (from cleared bits) repeat until a run makes no move.
// Here each round evaluates a window of blockDim consecutive cities in
// parallel against the current tour and applies the lowest-index improving
// move; the window's earlier cities had no move, so they get their bits set.
// That is exactly the sequential search, move for move, for any window size.
// A move reverses the shorter of the two paths it cuts, with all threads.
//
// Neighbour lists are the colony's candidate lists.  Distances are the exact
// integer ones (coordinates or the explicit matrix).
#include <climits>

#include "internal.cuh"

namespace mmas {

namespace {

template <bool XY>
__device__ __forceinline__ int32_t dij(const TwoOptArgs &a, int u, int v)
{
    if constexpr (XY)
        return euc2d_exact(__ldg(a.xy + u), __ldg(a.xy + v));
    else
        return __ldg(a.dist + (size_t)u * a.ld + v);
}

// First improving move at city c1: successor side, then predecessor side,
// neighbours in list order while closer than the tour neighbour on that side.
// mv = {u1, v1, u2, v2}: remove u1->v1 and u2->v2, add u1-u2 and v1-v2.
template <bool XY>
__device__ __forceinline__ bool find_move(const TwoOptArgs &a, const int32_t *tour,
                                          const int32_t *pos, int c1, int mv[4])
{
    const int n = a.n;
    const int p = pos[c1];
    const int s1 = tour[p + 1 == n ? 0 : p + 1], p1 = tour[p == 0 ? n - 1 : p - 1];
    const int32_t *nn = a.nn + (size_t)c1 * a.k;
    int radius = dij<XY>(a, c1, s1);
    for (int h = 0; h < a.k; ++h) {
        const int c2 = __ldg(nn + h);
        const int d12 = dij<XY>(a, c1, c2);
        if (d12 >= radius) break;
        const int q = pos[c2];
        const int s2 = tour[q + 1 == n ? 0 : q + 1];
        const long long gain =
            (long long)radius + dij<XY>(a, c2, s2) - d12 - dij<XY>(a, s1, s2);
        if (gain > 0) {
            mv[0] = c1; mv[1] = s1; mv[2] = c2; mv[3] = s2;
            return true;
        }
    }
    radius = dij<XY>(a, p1, c1);
    for (int h = 0; h < a.k; ++h) {
        const int c2 = __ldg(nn + h);
        const int d12 = dij<XY>(a, c1, c2);
        if (d12 >= radius) break;
        const int q = pos[c2];
        const int p2 = tour[q == 0 ? n - 1 : q - 1];
        const long long gain =
            (long long)radius + dij<XY>(a, p2, c2) - d12 - dij<XY>(a, p1, p2);
        if (gain > 0) {
            mv[0] = p2; mv[1] = c2; mv[2] = p1; mv[3] = c1;
            return true;
        }
    }
    return false;
}

template <bool XY, bool IB>
__global__ void __launch_bounds__(1024) k_two_opt(const TwoOptArgs a)
{
    extern __shared__ __align__(16) int32_t sm[];
    const int n = a.n, tid = threadIdx.x, W = blockDim.x;
    int32_t *s_tour = sm, *s_pos = sm + n;
    unsigned char *s_dlb = reinterpret_cast<unsigned char *>(sm + 2 * n);
    __shared__ int s_first, s_red[32];
    __shared__ unsigned long long s_best;
    __shared__ int s_mv[4];

    int first_tour = blockIdx.x, tour_step = gridDim.x;
    if constexpr (IB) {
        // the iteration best: shortest tour, ties -> lower ant
        unsigned long long best = ~0ull;
        for (int k = tid; k < a.m; k += W) {
            const unsigned long long key =
                ((unsigned long long)(uint32_t)a.lens[k] << 32) | (uint32_t)k;
            best = key < best ? key : best;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xFFFFFFFFu, best, o);
            best = w < best ? w : best;
        }
        if (tid == 0) s_best = ~0ull;
        __syncthreads();
        if ((tid & 31) == 0) atomicMin(&s_best, best);
        __syncthreads();
        first_tour = (int)(s_best & 0xFFFFFFFFull);
    }

    for (int ti = first_tour; ti < a.m; ti = IB ? a.m : ti + tour_step) {
        int32_t *row = a.tours + (size_t)ti * a.ld;
        for (int i = tid; i < n; i += W) {
            const int c = row[i];
            s_tour[i] = c;
            s_pos[c] = i;
        }
        __syncthreads();
        // every move shortens the tour by >= 1, so the search ends; the cap
        // (far above the moves a tour needs) only guards against a defect
        const long long cap = 64LL * n;
        long long total = 0;
        bool capped = false;
        for (;;) {  // runs
            for (int i = tid; i < n; i += W) s_dlb[i] = 0;
            __syncthreads();
            long long run_moves = 0;
            bool improved = true;
            while (improved && !capped) {  // passes
                improved = false;
                int l = 0;
                while (l < n) {  // windows
                    const int c1 = l + tid;
                    int mv[4];
                    const bool has = c1 < n && !s_dlb[c1] && find_move<XY>(a, s_tour, s_pos, c1, mv);
                    if (tid == 0) s_first = INT_MAX;
                    __syncthreads();
                    if (has) atomicMin(&s_first, c1);
                    __syncthreads();
                    const int first = s_first;
                    if (first == INT_MAX) {
                        if (c1 < n) s_dlb[c1] = 1;
                        l += W;
                        __syncthreads();
                        continue;
                    }
                    if (c1 < first) s_dlb[c1] = 1;  // evaluated, no move
                    if (c1 == first) {
                        s_mv[0] = mv[0]; s_mv[1] = mv[1]; s_mv[2] = mv[2]; s_mv[3] = mv[3];
                    }
                    __syncthreads();
                    const int u1 = s_mv[0], v1 = s_mv[1], u2 = s_mv[2], v2 = s_mv[3];
                    int pa = s_pos[v1], pb = s_pos[u2];
                    int len = (pb - pa + n) % n + 1;
                    if (2 * len > n) {  // reverse the complementary, shorter path
                        pa = s_pos[v2];
                        pb = s_pos[u1];
                        len = n - len;
                    }
                    __syncthreads();  // every thread has read the positions
                    for (int s = tid; s < len / 2; s += W) {
                        const int i = (pa + s) % n, j = (pb - s + n) % n;
                        const int ci = s_tour[i], cj = s_tour[j];
                        s_tour[i] = cj;
                        s_pos[cj] = i;
                        s_tour[j] = ci;
                        s_pos[ci] = j;
                    }
                    __syncthreads();
                    if (tid == 0) {
                        s_dlb[u1] = 0; s_dlb[v1] = 0; s_dlb[u2] = 0; s_dlb[v2] = 0;
                    }
                    improved = true;
                    ++run_moves;
                    l = first + 1;
                    __syncthreads();
                    if (++total > cap) {
                        if (tid == 0) atomicOr(a.err, ERR_LS_CAP);
                        capped = true;
                        break;
                    }
                }
            }
            if (run_moves == 0 || capped) break;
        }
        // write back and measure the improved tour
        int part = 0;
        for (int i = tid; i < n; i += W) {
            const int u = s_tour[i], v = s_tour[i + 1 == n ? 0 : i + 1];
            row[i] = u;
            part += dij<XY>(a, u, v);
        }
        part = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)part);
        if ((tid & 31) == 0) s_red[tid >> 5] = part;
        __syncthreads();
        if (tid == 0) {
            int sum = 0;
            for (int w = 0; w < (W >> 5); ++w) sum += s_red[w];
            a.lens[ti] = sum;
        }
        __syncthreads();
    }
}

}  // namespace

size_t two_opt_smem(int n) { return (size_t)9 * n + 16; }

cudaError_t launch_two_opt(const TwoOptArgs &a, bool iteration_best, int num_sms, cudaStream_t s)
{
    const size_t smem = two_opt_smem(a.n);
    const void *fn;
    int threads, grid;
    if (iteration_best) {
        fn = a.xy ? (const void *)k_two_opt<true, true> : (const void *)k_two_opt<false, true>;
        threads = 1024;
        grid = 1;
    } else {
        fn = a.xy ? (const void *)k_two_opt<true, false> : (const void *)k_two_opt<false, false>;
        threads = 256;
        grid = a.m < num_sms * 8 ? a.m : num_sms * 8;
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (iteration_best) {
        if (a.xy) k_two_opt<true, true><<<grid, threads, smem, s>>>(a);
        else k_two_opt<false, true><<<grid, threads, smem, s>>>(a);
    } else {
        if (a.xy) k_two_opt<true, false><<<grid, threads, smem, s>>>(a);
        else k_two_opt<false, false><<<grid, threads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace mmas
