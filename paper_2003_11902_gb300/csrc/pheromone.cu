// The rest of an iteration after construction (Alg. 1; Sec. 2.1, Sec. 4.4):
//   k_score   tour lengths (exact integer distances, one CTA per ant), then
//             in its last CTA:
//   select_best  iteration best (shortest tour, ties -> lower ant), global best
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

#include "distance.cuh"
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

// Iteration best, global best, limits, deposit amount and the deposited tour's
// neighbours; run by ONE CTA (any multiple of 32 threads up to 1024).  Two
// dependent memory rounds: the lengths (and the current global best), then the
// chosen tour, which is copied and turned into neighbours in the same pass.
__device__ void select_best(const BestArgs &a)
{
    __shared__ unsigned long long red[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    Scalars *sc = a.sc;
    const int gb = *((volatile int *)&sc->gb_len);
    unsigned long long best = ~0ull;
    for (int k = tid; k < a.m; k += blockDim.x) {
        const unsigned long long key =
            ((unsigned long long)(uint32_t)__ldcg(a.lens + k) << 32) | (uint32_t)k;
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
    const bool improved = len < gb;

    // deposit on the iteration best, or on the global best (which is the
    // iteration best when it improved)
    const bool from_ib = a.deposit == 0 || improved;
    const int32_t *dep = from_ib ? a.tours + (size_t)ib * a.ld : a.gb_tour;
    for (int t = tid; t < a.n; t += blockDim.x) {
        const int v = dep[t];
        const int nx = dep[t + 1 == a.n ? 0 : t + 1];
        const int pv = dep[t == 0 ? a.n - 1 : t - 1];
        a.nbr[v] = make_int2(nx, pv);
        if (improved) a.gb_tour[t] = v;
    }
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
}

__global__ void __launch_bounds__(1024) k_best(const BestArgs a)
{
    if (a.skip && *a.skip) return;
    select_best(a);
}

// Length of one tour, summed by the whole CTA (the result is valid in thread
// 0).  Each thread takes four consecutive edges per round (an int4 of the tour
// plus the following node) and issues all of their loads before using them.
// Distances are the exact integer ones.
template <bool XY>
__device__ __forceinline__ int score_ant(const ScoreArgs &a, int ant, int *red)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t *tr = a.tours + (size_t)ant * a.ld;
    int part = 0;
    for (int q = tid; 4 * q < a.n; q += blockDim.x) {
        const int t0 = 4 * q;
        const int4 u4 = *reinterpret_cast<const int4 *>(tr + t0);  // ld is a multiple of 32
        const int nx = tr[t0 + 4 < a.n ? t0 + 4 : 0];
        const int node[5] = {u4.x, u4.y, u4.z, u4.w, nx};
        const int cnt = a.n - t0 < 4 ? a.n - t0 : 4;  // edges t0 .. t0+cnt-1
        // edge e joins node[e] and node[e+1]; the last real edge closes on nx
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (e >= cnt) break;
            const int from = node[e];
            const int to = (e + 1 < cnt) ? node[e + 1] : nx;
            if constexpr (XY)
                part += euc2d_exact(__ldg(a.xy + from), __ldg(a.xy + to));
            else
                part += __ldg(a.dist + (size_t)from * a.ld + to);
        }
    }
    part = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    int sum = 0;
    if (tid == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sum += red[i];
    __syncthreads();
    return sum;
}

// Tour lengths, then -- when a.best -- the last CTA to finish runs select_best
// on all m lengths.  One CTA per ant (looping when m exceeds the grid).
template <bool XY>
__global__ void __launch_bounds__(256) k_score(const ScoreArgs a)
{
    __shared__ int red[8];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    for (int ant = blockIdx.x; ant < a.m; ant += gridDim.x) {
        const int len = score_ant<XY>(a, ant, red);
        if (tid == 0) a.lens[ant] = len;
    }
    if (!a.best) return;
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&a.b.sc->done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    select_best(a.b);
    if (tid == 0) a.b.sc->done = 0;
}

// Batched lengths: one CTA per ant of every colony; the last CTA of a
// colony to finish runs that colony's select_best.
template <bool XY>
__global__ void __launch_bounds__(256)
    k_score_batch(const ScoreArgs *__restrict__ args, const int32_t *__restrict__ ant_colony,
                  const int32_t *__restrict__ ant_base)
{
    __shared__ int red[8];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const int b = ant_colony[blockIdx.x];
    const ScoreArgs a = args[b];
    const int ant = (int)blockIdx.x - ant_base[b];
    const int len = score_ant<XY>(a, ant, red);
    if (tid == 0) a.lens[ant] = len;
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&a.b.sc->done, 1u) == (unsigned)a.m - 1u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    select_best(a.b);
    if (tid == 0) a.b.sc->done = 0;
}

// Row i of the fused pass: evaporate with both clamps, deposit on the row's
// two tour edges, write choice_info (or its reciprocal), then gather
// 1/choice_info of the row's candidates.  The whole CTA works on the row.
// With a reach list (xe > 0) the pass also gathers the listed nodes'
// choice_info and takes the row's largest choice_info among the nodes j != i
// whose eta^beta does not exceed the last listed node's: every node outside
// the list is among them (eta^beta does not increase with distance beyond the
// list), so this bounds their choice_info for the greedy fallback.
template <bool FULLROW, bool ALPHA1, bool EXTRAS>
__device__ __forceinline__ void update_row_cta(const UpdateArgs &a, int i, float tmin, float tmax,
                                               float delta)
{
    __shared__ uint32_t s_bound[8], s_ball[8];
    __shared__ int s_nx, s_hot[8];
    const bool reach = !FULLROW && a.xe > 0;  // (no far list: n <= UPDATE_CTA_MAX_N)
    // the extra list (xhot set) is filled only for rows that had few nodes
    // above the trail floor outside the list at the last pass (that changes
    // slowly); the others just count theirs
    const bool extras = EXTRAS && reach && a.xhot != nullptr;
    const bool gather_hot = extras && a.xhot[i] <= 2 * REACH_EXTRA;
    if (gather_hot) {  // the same for the whole CTA
        if (threadIdx.x == 0) s_nx = 0;
        __syncthreads();
    }
    float bound_all = 0.0f;
    int hot_cnt = 0;
    // no node lies outside a list of all n - 1 others
    const float thr = (reach && a.xe < a.n - 1)
                          ? __ldg(a.eb + (size_t)i * a.ld + a.xl32[(size_t)i * a.xe + a.xe - 1])
                          : -1.0f;
    float bound = 0.0f;
    const int nq = a.ld >> 2;
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
            float w = 0.0f;
            if (j < a.n) {
                if (a.evaporate) {
                    x = fminf(fmaxf(__fmul_rn(x, a.persist), tmin), tmax);
                    if (j == succ || j == pred) x = fminf(__fadd_rn(x, delta), tmax);
                }
                w = ALPHA1 ? __fmul_rn(x, ev[c]) : __fmul_rn(powf(x, a.alpha), ev[c]);
                wv[c] = (FULLROW && a.recip) ? __frcp_rn(w) : w;
            } else {
                x = 0.0f;
                wv[c] = 0.0f;
            }
            tv[c] = x;
            if (!FULLROW && reach && j < a.n && j != i && ev[c] <= thr) {
                // outside the list: a node above the trail floor is stored while
                // room is left; `bound` covers the others, `bound_all` all
                bool stored = false;
                if (extras && x > tmin) {
                    ++hot_cnt;
                    if (gather_hot && *reinterpret_cast<volatile int *>(&s_nx) < REACH_EXTRA) {
                        const int slot = atomicAdd(&s_nx, 1);
                        if (slot < REACH_EXTRA) {
                            a.xxw[(size_t)i * REACH_EXTRA + slot] = make_uint2(__float_as_uint(w), (uint32_t)j);
                            stored = true;
                        }
                    }
                }
                if (!stored) bound = fmaxf(bound, w);
                if (EXTRAS) bound_all = fmaxf(bound_all, w);
            }
        }
        trow[q] = make_float4(tv[0], tv[1], tv[2], tv[3]);
        wrow[q] = make_float4(wv[0], wv[1], wv[2], wv[3]);
    }
    if (!FULLROW && a.cl > 0) {
        if (reach) {  // choice_info >= 0: its bits order like the values
            const uint32_t wmax = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(bound));
            if ((threadIdx.x & 31) == 0) s_bound[threadIdx.x >> 5] = wmax;
            if (extras) {
                const uint32_t amax = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(bound_all));
                const int hots = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)hot_cnt);
                if ((threadIdx.x & 31) == 0) {
                    s_ball[threadIdx.x >> 5] = amax;
                    s_hot[threadIdx.x >> 5] = hots;
                }
            }
        }
        __syncthreads();  // this row's choice_info is written and visible to the CTA
        const float *w1 = a.wmat + (size_t)i * a.ld;
        for (int c = threadIdx.x; c < a.cl; c += blockDim.x) {
            const int v = a.cand32[(size_t)i * a.cl + c];
            a.cwinv[(size_t)i * a.cl + c] = __frcp_rn(w1[v]);
        }
        if (reach) {
            for (int e = threadIdx.x; e < a.xe; e += blockDim.x) {
                const int v = a.xl32[(size_t)i * a.xe + e];
                a.xlw[(size_t)i * a.xe + e] = make_uint2(__float_as_uint(w1[v]), (uint32_t)v);
            }
            if (threadIdx.x == 0) {
                uint32_t m = 0, ma = 0;
                int hots = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    m = s_bound[w] > m ? s_bound[w] : m;
                    if (extras) {
                        ma = s_ball[w] > ma ? s_ball[w] : ma;
                        hots += s_hot[w];
                    }
                }
                // every node above the floor stored: the extra list is exact and
                // the bound covers the rest; else the list is unused (without
                // the extra list, bound already covers every outside node)
                const bool all = gather_hot && hots <= REACH_EXTRA;
                a.xlb[i] = __uint_as_float(all || !extras ? m : ma);
                a.xxn[i] = all ? hots : 0;
                if (extras) a.xhot[i] = hots;
            }
            __syncthreads();  // s_bound is read before the CTA's next row writes it
        }
    }
}

// One CTA per row: for colonies with few rows, where every row's latency counts.
template <bool FULLROW, bool ALPHA1>
__global__ void __launch_bounds__(256, 4) k_update_cta(const UpdateArgs a)
{
    if (a.skip && *a.skip) return;
    const float tmin = a.sc->tmin, tmax = a.sc->tmax, delta = a.sc->delta;
    for (int i = blockIdx.x; i < a.n; i += gridDim.x) update_row_cta<FULLROW, ALPHA1, true>(a, i, tmin, tmax, delta);
}

// The same pass with one warp per row (slots of the extra list by ballot),
// for colonies of many rows and for the batched pass: no CTA barrier, and the
// latency of a row is hidden by the other rows of the SM.
template <bool FULLROW, bool ALPHA1, bool EXTRAS>
__device__ __forceinline__ void update_row(const UpdateArgs &a, int i, float tmin, float tmax,
                                           float delta, int lane)
{
    const bool reach = !FULLROW && a.xe > 0;
    // the extra list (xhot set) is filled only for rows that had few nodes
    // above the trail floor outside the list at the last pass (that changes
    // slowly); the others just count theirs
    const bool extras = EXTRAS && reach && a.xhot != nullptr;
    const bool gather_hot = extras && a.xhot[i] <= 2 * REACH_EXTRA;
    // no node lies outside a list of all n - 1 others
    const float thr = (reach && a.xe < a.n - 1)
                          ? __ldg(a.eb + (size_t)i * a.ld + a.xl32[(size_t)i * a.xe + a.xe - 1])
                          : -1.0f;
    // far list: the bound covers every node j != i with eta^beta_ij at most that
    // of the row's last far node (every node beyond the list)
    const bool far = reach && a.fe > 0;
    const float thr_far = far ? __ldg(a.eb + (size_t)i * a.ld + a.xf16[(size_t)i * a.fp + a.fp - 1]) : -1.0f;
    float bound = 0.0f, bound_all = 0.0f, bound_far = 0.0f;
    int hot_cnt = 0, nx = 0;  // nx: extras stored so far (the same in every lane)
    const unsigned below = (1u << lane) - 1u;
    const int nq = a.ld >> 2;
    int succ = -1, pred = -1;
    if (a.nbr) {
        const int2 nb = a.nbr[i];
        succ = nb.x;
        pred = nb.y;
    }
    float4 *trow = reinterpret_cast<float4 *>(a.tau + (size_t)i * a.ld);
    const float4 *erow = reinterpret_cast<const float4 *>(a.eb + (size_t)i * a.ld);
    float4 *wrow = reinterpret_cast<float4 *>(a.wmat + (size_t)i * a.ld);
    // the next round's loads are issued before this round's arithmetic, so a
    // warp keeps two rounds of the row in flight
    float4 t4n = lane < nq ? trow[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 e4n = lane < nq ? __ldg(erow + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q0 = 0; q0 < nq; q0 += 32) {  // every lane takes each round
        const int q = q0 + lane;
        const bool inq = q < nq;
        const float4 t4 = t4n;
        const float4 e4 = e4n;
        if (q + 32 < nq) {
            t4n = trow[q + 32];
            e4n = __ldg(erow + q + 32);
        }
        float tv[4] = {t4.x, t4.y, t4.z, t4.w};
        const float ev[4] = {e4.x, e4.y, e4.z, e4.w};
        float wv[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = (q << 2) + c;
            float x = tv[c];
            float w = 0.0f;
            if (j < a.n) {
                if (a.evaporate) {
                    x = fminf(fmaxf(__fmul_rn(x, a.persist), tmin), tmax);
                    if (j == succ || j == pred) x = fminf(__fadd_rn(x, delta), tmax);
                }
                w = ALPHA1 ? __fmul_rn(x, ev[c]) : __fmul_rn(powf(x, a.alpha), ev[c]);
                wv[c] = (FULLROW && a.recip) ? __frcp_rn(w) : w;
            } else {
                x = 0.0f;
                wv[c] = 0.0f;
            }
            tv[c] = x;
            if (!FULLROW && reach) {
                // outside the list: a node above the trail floor is stored while
                // room is left (slots by warp ballot); `bound` covers the
                // others, `bound_all` all of them
                const bool outside = j < a.n && j != i && ev[c] <= thr;
                const bool hot = extras && outside && x > tmin;
                hot_cnt += hot ? 1 : 0;
                bool stored = false;
                if (gather_hot) {  // the same in every lane
                    const unsigned hm = __ballot_sync(0xFFFFFFFFu, hot);
                    if (hot) {
                        const int slot = nx + __popc(hm & below);
                        if (slot < REACH_EXTRA) {
                            a.xxw[(size_t)i * REACH_EXTRA + slot] = make_uint2(__float_as_uint(w), (uint32_t)j);
                            stored = true;
                        }
                    }
                    nx += __popc(hm);
                }
                if (outside && !stored) bound = fmaxf(bound, w);
                if (EXTRAS && outside) bound_all = fmaxf(bound_all, w);
                if (far && outside && ev[c] <= thr_far) bound_far = fmaxf(bound_far, w);
            }
        }
        if (inq) {
            trow[q] = make_float4(tv[0], tv[1], tv[2], tv[3]);
            wrow[q] = make_float4(wv[0], wv[1], wv[2], wv[3]);
        }
    }
    if (!FULLROW && a.cl > 0) {
        __syncwarp();  // the row's choice_info, written by this warp, is visible to its lanes
        const float *w1 = a.wmat + (size_t)i * a.ld;
        for (int c = lane; c < a.cl; c += 32) {
            const int v = a.cand32[(size_t)i * a.cl + c];
            a.cwinv[(size_t)i * a.cl + c] = __frcp_rn(w1[v]);
        }
        if (reach) {
            for (int e = lane; e < a.xe; e += 32) {
                const int v = a.xl32[(size_t)i * a.xe + e];
                a.xlw[(size_t)i * a.xe + e] = make_uint2(__float_as_uint(w1[v]), (uint32_t)v);
            }
            // choice_info >= 0: its bits order like the values
            const uint32_t m = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(bound));
            const uint32_t ma = extras ? __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(bound_all)) : 0u;
            const int hots = extras ? (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)hot_cnt) : 0;
            const uint32_t mf = far ? __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(bound_far)) : 0u;
            if (lane == 0) {
                // every node above the floor stored: the extra list is exact and
                // the bound covers the rest; else the list is unused (without
                // the extra list, bound already covers every outside node)
                const bool all = gather_hot && hots <= REACH_EXTRA;
                a.xlb[i] = __uint_as_float(all || !extras ? m : ma);
                a.xxn[i] = all ? hots : 0;
                if (extras) a.xhot[i] = hots;
                if (far) a.xfb[i] = __uint_as_float(mf);
            }
        }
    }
}

// One warp per row, eight rows per CTA.
template <bool FULLROW, bool ALPHA1>
__global__ void __launch_bounds__(256, 4) k_update(const UpdateArgs a)
{
    if (a.skip && *a.skip) return;
    const float tmin = a.sc->tmin, tmax = a.sc->tmax, delta = a.sc->delta;
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < a.n; i += nwarps)
        update_row<FULLROW, ALPHA1, true>(a, i, tmin, tmax, delta, lane);
}

// Batched fused pass: one warp per row of every colony.
template <bool ALPHA1>
__global__ void __launch_bounds__(256, 4)
    k_update_batch(const UpdateArgs *__restrict__ args, const int32_t *__restrict__ row_colony,
                   const int32_t *__restrict__ row_base, int total_rows)
{
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= total_rows) return;
    const int b = row_colony[row];
    const UpdateArgs a = args[b];
    update_row<false, ALPHA1, false>(a, row - row_base[b], a.sc->tmin, a.sc->tmax, a.sc->delta,
                                     threadIdx.x & 31);
}

}  // namespace

cudaError_t launch_best(const BestArgs &a, cudaStream_t s)
{
    k_best<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_score(const ScoreArgs &a, int num_sms, cudaStream_t s)
{
    // one CTA per ant, at most 16 resident per SM's worth; CTAs loop over ants
    int grid = a.m < num_sms * 8 ? a.m : num_sms * 8;
    if (a.xy)
        k_score<true><<<grid, 256, 0, s>>>(a);
    else
        k_score<false><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_score_batch(const ScoreArgs *args, const int32_t *ant_colony, const int32_t *ant_base,
                               int total_ants, bool xy, cudaStream_t s)
{
    if (xy)
        k_score_batch<true><<<total_ants, 256, 0, s>>>(args, ant_colony, ant_base);
    else
        k_score_batch<false><<<total_ants, 256, 0, s>>>(args, ant_colony, ant_base);
    return cudaGetLastError();
}

cudaError_t launch_update_batch(const UpdateArgs *args, const int32_t *row_colony, const int32_t *row_base,
                                int total_rows, bool alpha1, cudaStream_t s)
{
    const int grid = (total_rows + 7) / 8;
    if (alpha1)
        k_update_batch<true><<<grid, 256, 0, s>>>(args, row_colony, row_base, total_rows);
    else
        k_update_batch<false><<<grid, 256, 0, s>>>(args, row_colony, row_base, total_rows);
    return cudaGetLastError();
}

cudaError_t launch_update(const UpdateArgs &a, int num_sms, cudaStream_t s)
{
    const bool a1 = a.alpha == 1.0f;
    if (a.n <= UPDATE_CTA_MAX_N) {  // a CTA per row: few rows, each one's latency counts
        const int grid = a.n < num_sms * 8 ? a.n : num_sms * 8;
        if (a.fullrow) {
            if (a1) k_update_cta<true, true><<<grid, 256, 0, s>>>(a);
            else k_update_cta<true, false><<<grid, 256, 0, s>>>(a);
        } else {
            if (a1) k_update_cta<false, true><<<grid, 256, 0, s>>>(a);
            else k_update_cta<false, false><<<grid, 256, 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    const int rows8 = (a.n + 7) / 8;  // eight rows (warps) per CTA
    const int grid = rows8 < num_sms * 8 ? rows8 : num_sms * 8;
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
