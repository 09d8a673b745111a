// 2-opt local search (Sec. 5.7): Bentley's neighbour-list 2-opt with
// don't-look bits, first improvement, on whole tours.
//
// One CTA improves one tour held in shared memory (tour and position of each
// city, the length of each tour edge, don't-look bits: 13 bytes per city).
// The sequential search visits the cities in index order, skipping those
// whose don't-look bit is set; a city
// without a move gets its bit set, a move clears the bits of its four cities
// and the visit continues after the moving city; a run ends after a pass with
// no move, and runs (from cleared bits) repeat until a run makes no move.
// Here each round evaluates a window of consecutive cities in parallel against
// the current tour and applies the lowest-index improving move; the window's
// earlier cities had no move, so they get their bits set.  That is exactly the
// sequential search, move for move, for any window size: the window is 32
// cities after a move (moves come densely) and doubles, up to blockDim, while
// windows find none.  A move reverses the shorter of the two paths it cuts,
// with all threads.
//
// Neighbour lists are the colony's candidate lists, with their distances
// precomputed.  Distances are the exact integer ones (coordinates or the
// explicit matrix).
#include <climits>

#include "internal.cuh"
#include "twoopt.cuh"

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

// Shared-memory image of one tour: tour[i], pos[c], and
// edge[i] = d(tour[i], tour[i+1 mod n]) kept exact under every move.
struct TourView {
    int32_t *tour, *pos;
    int32_t *edge;
    int n;
    __device__ __forceinline__ int nxt(int i) const { return i + 1 == n ? 0 : i + 1; }
    __device__ __forceinline__ int prv(int i) const { return i == 0 ? n - 1 : i - 1; }
};

// First improving move at city c1: successor side, then predecessor side,
// neighbours in list order while closer than the tour neighbour on that side.
// mv = {u1, v1, u2, v2}: remove u1->v1 and u2->v2, add u1-u2 and v1-v2.
// Tour-edge lengths come from the edge array, neighbour distances from the
// precomputed lists; one distance is computed per neighbour examined.
template <bool XY>
__device__ __forceinline__ bool find_move(const TwoOptArgs &a, const TourView &tv, int c1,
                                          int mv[4])
{
    const int p = tv.pos[c1];
    const int s1 = tv.tour[tv.nxt(p)], p1 = tv.tour[tv.prv(p)];
    const int32_t *nn = a.nn + (size_t)c1 * a.k;
    const int32_t *dn = a.nnd + (size_t)c1 * a.k;
    int radius = tv.edge[p];
    for (int h = 0; h < a.k; ++h) {
        const int d12 = __ldg(dn + h);
        if (d12 >= radius) break;
        const int c2 = __ldg(nn + h);
        const int q = tv.pos[c2];
        const int s2 = tv.tour[tv.nxt(q)];
        const long long gain = (long long)radius + tv.edge[q] - d12 - dij<XY>(a, s1, s2);
        if (gain > 0) {
            mv[0] = c1; mv[1] = s1; mv[2] = c2; mv[3] = s2;
            return true;
        }
    }
    radius = tv.edge[tv.prv(p)];
    for (int h = 0; h < a.k; ++h) {
        const int d12 = __ldg(dn + h);
        if (d12 >= radius) break;
        const int c2 = __ldg(nn + h);
        const int q = tv.pos[c2];
        const int p2 = tv.tour[tv.prv(q)];
        const long long gain = (long long)radius + tv.edge[tv.prv(q)] - d12 - dij<XY>(a, p1, p2);
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
    TourView tv;
    tv.n = n;
    tv.edge = sm;
    tv.tour = sm + n;
    tv.pos = sm + 2 * n;
    unsigned char *s_dlb = reinterpret_cast<unsigned char *>(tv.pos + n);
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
            tv.tour[i] = c;
            tv.pos[c] = i;
            tv.edge[i] = dij<XY>(a, c, row[i + 1 == n ? 0 : i + 1]);
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
                int w = 32;  // window: 32 cities after a move, doubling while none is found
                while (l < n) {  // windows
                    const int c1 = l + tid;
                    const bool in = tid < w && c1 < n;
                    int mv[4];
                    const bool has = in && !s_dlb[c1] && find_move<XY>(a, tv, c1, mv);
                    if (tid == 0) s_first = INT_MAX;
                    __syncthreads();
                    if (has) atomicMin(&s_first, c1);
                    __syncthreads();
                    const int first = s_first;
                    if (first == INT_MAX) {
                        if (in) s_dlb[c1] = 1;
                        l += w;
                        w = w * 2 < W ? w * 2 : W;
                        __syncthreads();
                        continue;
                    }
                    w = 32;
                    if (in && c1 < first) s_dlb[c1] = 1;  // evaluated, no move
                    if (c1 == first) {
                        s_mv[0] = mv[0]; s_mv[1] = mv[1]; s_mv[2] = mv[2]; s_mv[3] = mv[3];
                    }
                    __syncthreads();
                    const int u1 = s_mv[0], v1 = s_mv[1], u2 = s_mv[2], v2 = s_mv[3];
                    int pa = tv.pos[v1], pb = tv.pos[u2];
                    int len = (pb - pa + n) % n + 1;
                    if (2 * len > n) {  // reverse the complementary, shorter path
                        pa = tv.pos[v2];
                        pb = tv.pos[u1];
                        len = n - len;
                    }
                    __syncthreads();  // every thread has read the positions
                    // reverse tour[pa..pb]; the len-1 edges inside it reverse too
                    for (int s2 = tid; s2 < len / 2; s2 += W) {
                        const int i = (pa + s2) % n, j = (pb - s2 + n) % n;
                        const int ci = tv.tour[i], cj = tv.tour[j];
                        tv.tour[i] = cj;
                        tv.pos[cj] = i;
                        tv.tour[j] = ci;
                        tv.pos[ci] = j;
                    }
                    for (int s2 = tid; s2 < (len - 1) / 2; s2 += W) {
                        const int i = (pa + s2) % n, j = (pb - 1 - s2 + n) % n;
                        const int ei = tv.edge[i];
                        tv.edge[i] = tv.edge[j];
                        tv.edge[j] = ei;
                    }
                    __syncthreads();
                    if (tid == 0) {
                        s_dlb[u1] = 0; s_dlb[v1] = 0; s_dlb[u2] = 0; s_dlb[v2] = 0;
                        // the two added edges now border the reversed path
                        const int ia = tv.prv(pa);
                        tv.edge[ia] = dij<XY>(a, tv.tour[ia], tv.tour[pa]);
                        tv.edge[pb] = dij<XY>(a, tv.tour[pb], tv.tour[tv.nxt(pb)]);
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
            row[i] = tv.tour[i];
            part += tv.edge[i];
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

// d(c, nn[c][h]) for every city and neighbour (set-up, once).
template <bool XY>
__global__ void k_neighbour_dist(const TwoOptArgs a, int32_t *nnd)
{
    const size_t total = (size_t)a.n * a.k;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / a.k);
        nnd[e] = dij<XY>(a, c, a.nn[e]);
    }
}

}  // namespace

size_t two_opt_smem(int n) { return (size_t)13 * n + 16; }

cudaError_t launch_neighbour_dist(const TwoOptArgs &a, int32_t *nnd, cudaStream_t s)
{
    if (a.xy)
        k_neighbour_dist<true><<<256, 256, 0, s>>>(a, nnd);
    else
        k_neighbour_dist<false><<<256, 256, 0, s>>>(a, nnd);
    return cudaGetLastError();
}

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
