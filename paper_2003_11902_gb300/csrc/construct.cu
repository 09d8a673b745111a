// Solution construction (Alg. 1, inner loops).
//
// One warp builds one ant's tour.  At each of the n-1 steps the warp scores the
// unvisited nodes of Eq. (1)'s neighbourhood with weighted-reservoir keys
// log2(r) / w (Alg. 4, Sec. 4.2.2), reduces them with one redux.max and one
// redux.min (ties -> lower node id), marks the winner in a bitmask tabu
// (Sec. 4.1) and appends it to the tour.  Tour lengths are computed afterwards
// by the scoring kernel, off this dependency chain.
//
//  - Candidate-list mode (cl in 1..32, Sec. 4.3): lane c scores candidate
//    slot c.  A slot's uniform depends on (iteration, ant, step, slot) only, so
//    one Philox call yields the draws of four consecutive steps; the call for
//    the next four steps and its log2s are spread over the current four steps.
//    When every candidate is visited, an out-of-line fallback scans the row.
//  - Whole-row mode (cl = 0): lane l scores nodes 4c..4c+3 for c = l, l+32, ...,
//    reading 16 bytes of 1/choice_info per chunk, one Philox call per chunk.
//
// The table a step reads (n x cl ids + reciprocal weights, or the n x ld
// reciprocal weight matrix) is copied into shared memory once per CTA with the
// bulk-copy engine when it fits; each CTA then runs ceil(m / #SMs) ants.
// The tabu of an ant lives in registers (lane l holds nodes 32l..32l+31) when
// n <= 1024, otherwise in the warp's slice of shared memory.  Tour entries are
// buffered one per lane and written as 128-byte rows every 32 steps.
#include "internal.cuh"

namespace mmas {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr unsigned long long STAGE_LIMIT_NS = 2000000000ull;  // 2 s
constexpr unsigned long long EXPIRE_LIMIT_NS = 1000000ull;    // 1 ms

// Testing aid (mmas_debug_expire_stage_waits): when set, every staging first
// waits for g_never_set, which nothing writes, until its 1 ms limit runs out,
// and then takes the timeout path.
__device__ uint32_t g_expire_stage_waits;
__device__ uint32_t g_never_set;
constexpr uint32_t BULK_CHUNK = 32768u;

enum { CAND = 0, ROW = 1 };

// Bitmask tabu (Sec. 4.1, "BT"): mark / is_visited in O(1).  TW = 1, 2 or 4:
// the bitmask lives in registers, lane l holding words l, l + 32, ... (n up to
// 1024 TW nodes); TW = 0: in the warp's slice of shared memory.
template <int TW>
struct Tabu {
    static constexpr int R = TW > 0 ? TW : 1;
    uint32_t reg[R];           // TW > 0: words lane, lane + 32, ...
    uint32_t *w = nullptr;     // TW = 0: this warp's words in shared memory
    int nw = 0;

    __device__ __forceinline__ void clear(int lane)
    {
        if constexpr (TW > 0) {
#pragma unroll
            for (int j = 0; j < R; ++j) reg[j] = 0;
        } else {
            for (int q = lane; q < nw; q += 32) w[q] = 0;
            __syncwarp();
        }
    }
    // Mark node v when `on` (warp-uniform).  Registers: selects, not a branch
    // (a one-lane branch diverges the warp).
    __device__ __forceinline__ void mark_if(int lane, int v, bool on)
    {
        if constexpr (TW > 0) {
            const int q = v >> 5;
#pragma unroll
            for (int j = 0; j < R; ++j) reg[j] |= (on && q == lane + 32 * j) ? (1u << (v & 31)) : 0u;
        } else {
            if (on) {
                if (lane == 0) w[v >> 5] |= 1u << (v & 31);
                __syncwarp();
            }
        }
    }
    __device__ __forceinline__ void mark(int lane, int v) { mark_if(lane, v, true); }
    // The bitmask word that holds node v.  Every lane of the warp must call it.
    __device__ __forceinline__ uint32_t word_of(int v) const
    {
        if constexpr (TW == 0) {
            return w[v >> 5];
        } else if constexpr (TW == 1) {
            return __shfl_sync(FULL, reg[0], (v >> 5) & 31);
        } else {
            const int src = (v >> 5) & 31, j = (v >> 10) & (TW - 1);
            uint32_t x[R];
#pragma unroll
            for (int i = 0; i < R; ++i) x[i] = __shfl_sync(FULL, reg[i], src);
            uint32_t r = x[0];
#pragma unroll
            for (int i = 1; i < R; ++i) r = j == i ? x[i] : r;
            return r;
        }
    }
};

// Register words per lane for an n-node tabu, 0 when it must live in shared memory.
__host__ __device__ __forceinline__ int tabu_words(int n)
{
    return n <= 1024 ? 1 : (n <= 2048 ? 2 : (n <= 4096 ? 4 : 0));
}

__device__ __forceinline__ uint32_t pick_word(const uint4 &r, int e)
{
    return e == 0 ? r.x : (e == 1 ? r.y : (e == 2 ? r.z : r.w));
}

__device__ __forceinline__ float pick_f(const float4 &r, int e)
{
    return e == 0 ? r.x : (e == 1 ? r.y : (e == 2 ? r.z : r.w));
}

// Score every unvisited node of `row` in 4-node chunks and return the winner
// (ties -> lower id).  GREEDY: the key is the weight itself (the candidate-list
// fallback on choice_info); otherwise the reservoir key log2(r) * inv-weight,
// r from the whole-row stream, with `row` holding the reciprocal weights (RECIP)
// or the weights.  Eight chunk-columns (1024 nodes) are loaded before use, so
// rows of up to 1024 nodes cost one memory round trip.  The fallback scans
// (!RECIP: `row` is a row of choice_info in global memory) use streaming
// loads (evict-first): a scanned row is read once, and should not push the
// candidate rows the regular steps read out of L2.  The whole-row steps
// (RECIP) use generic loads: their table may be staged in shared memory, which
// a global-space load must not be given.
template <int TW, bool GREEDY, bool RECIP>
__device__ __forceinline__ int scan_row(const float *__restrict__ row, int n, const Tabu<TW> &tb,
                                        int lane, uint32_t t, uint32_t ant, uint32_t it,
                                        uint32_t k0, uint32_t k1, uint32_t *err, int cur)
{
    constexpr int U = 8;
    const int nch = (n + 3) >> 2;
    uint32_t bk = 0, bv = 0xFFFFFFFFu;
    for (int c0 = 0; c0 < nch; c0 += 32 * U) {
        float4 w4[U];
        uint32_t bits[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = c0 + 32 * u + lane;
            const int v0 = c << 2;
            const int vq = v0 < n ? v0 : n - 1;
            const uint32_t word = tb.word_of(vq);
            bits[u] = c < nch ? (word >> (v0 & 31)) & 0xFu : 0xFu;
            // a chunk whose four nodes are visited is not read
            const float4 *src = reinterpret_cast<const float4 *>(row + v0);
            if (c < nch && bits[u] != 0xFu)
                w4[u] = RECIP ? *src : __ldcs(src);
            else
                w4[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (bits[u] == 0xFu) continue;
            const int v0 = (c0 + 32 * u + lane) << 2;
            uint4 r = make_uint4(0u, 0u, 0u, 0u);
            if constexpr (!GREEDY) {
                r = make_uint4(0x80000000u | (uint32_t)(v0 >> 2), t, ant, it);
                philox_rounds<0, 10>(r, k0, k1);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int v = v0 + e;
                if (v >= n || ((bits[u] >> e) & 1u)) continue;
                const float x = pick_f(w4[u], e);
                uint32_t kk;
                if constexpr (GREEDY) {
                    kk = ord_key(x);
                } else {
                    const float lg = log2f(unit_open(pick_word(r, e)));
                    kk = ord_key(__fmul_rn(lg, RECIP ? x : __frcp_rn(x)));
                }
                if (kk > bk) {
                    bk = kk;
                    bv = (uint32_t)v;
                }
            }
        }
    }
    const uint32_t mx = __reduce_max_sync(FULL, bk);
    if (mx == 0u) {
        if (lane == 0) atomicOr(err, ERR_NO_UNVISITED);
        return cur;
    }
    return (int)__reduce_min_sync(FULL, bk == mx ? bv : 0xFFFFFFFFu);
}

// The same selection as scan_row over a row of which at most a few hundred
// nodes are unvisited, for tabus in shared memory: lane l walks the tabu words
// l, l + 32, ... and reads the weights of their unvisited nodes only, eight at
// a time per lane, so a late-tour scan costs a round trip or two and n - t
// sectors instead of the whole row.  Ties -> lower id (compared explicitly,
// the nodes are not visited in id order).
constexpr int SPARSE_SCAN_MAX = 1024;  // unvisited nodes below which the sparse form is used

template <bool GREEDY>
__device__ __forceinline__ int scan_unvisited(const float *__restrict__ row, int n, const uint32_t *tabu,
                                              int lane, uint32_t t, uint32_t ant, uint32_t it,
                                              uint32_t k0, uint32_t k1, uint32_t *err, int cur)
{
    constexpr int U = 8;
    const int nw = (n + 31) >> 5;
    const uint32_t tail = (n & 31) ? (1u << (n & 31)) - 1u : 0xFFFFFFFFu;
    uint32_t bk = 0u, bv = 0xFFFFFFFFu;
    int q = lane;
    uint32_t pend = q < nw ? ~tabu[q] & (q == nw - 1 ? tail : 0xFFFFFFFFu) : 0u;
    for (;;) {
        int vs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            while (pend == 0u && q < nw) {
                q += 32;
                pend = q < nw ? ~tabu[q] & (q == nw - 1 ? tail : 0xFFFFFFFFu) : 0u;
            }
            if (pend != 0u) {
                vs[u] = (q << 5) + __ffs(pend) - 1;
                pend &= pend - 1u;
            } else {
                vs[u] = -1;
            }
        }
        if (!__any_sync(FULL, vs[0] >= 0)) break;
        float x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = vs[u] >= 0 ? __ldcs(row + vs[u]) : 0.0f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (vs[u] < 0) continue;
            const uint32_t v = (uint32_t)vs[u];
            uint32_t kk;
            if constexpr (GREEDY) {
                kk = ord_key(x[u]);
            } else {
                uint4 r = make_uint4(0x80000000u | (v >> 2), t, ant, it);
                philox_rounds<0, 10>(r, k0, k1);
                kk = ord_key(__fmul_rn(log2f(unit_open(pick_word(r, (int)(v & 3u)))), __frcp_rn(x[u])));
            }
            if (kk > bk || (kk == bk && v < bv)) {
                bk = kk;
                bv = v;
            }
        }
    }
    const uint32_t mx = __reduce_max_sync(FULL, bk);
    if (mx == 0u) {
        if (lane == 0) atomicOr(err, ERR_NO_UNVISITED);
        return cur;
    }
    return (int)__reduce_min_sync(FULL, bk == mx ? bv : 0xFFFFFFFFu);
}

// The greedy fallback decided on cur's reach list: its REACH_MAX nearest nodes
// (fewer when n is small) and up to REACH_EXTRA other nodes whose trail is
// above tau_min, with this iteration's choice_info, and `bound`, the largest
// choice_info of any other node.  When the best unvisited node of the lists
// beats the bound strictly, every node of the row's largest choice_info is
// listed, so the listed winner (ties -> lower id) is the row's greedy choice;
// otherwise -1 and the caller scans the row.  One memory round trip: lane l
// holds entries l, l + 32, l + 64, l + 96 of the reach list and entry l of
// the extra list.
template <int TW>
__device__ __forceinline__ void reach_entry(uint2 e, bool in, const Tabu<TW> &tb, uint32_t &bk, uint32_t &bv)
{
    const uint32_t v = e.y;
    const uint32_t word = tb.word_of((int)v);  // every lane calls it
    const bool ok = in && !((word >> (v & 31)) & 1u);
    const uint32_t k = ok ? (e.x | 0x80000000u) : 0u;  // ord_key of choice_info >= 0
    if (k > bk || (k == bk && k != 0u && v < bv)) {
        bk = k;
        bv = v;
    }
}

template <int TW>
__device__ __forceinline__ int greedy_reach(const uint2 *__restrict__ xl, const float *__restrict__ xb,
                                            int xe, const uint2 *__restrict__ xx, const int32_t *xn,
                                            const Tabu<TW> &tb, int lane, uint32_t &mx_out,
                                            uint32_t &v_out)
{
    constexpr int P = REACH_MAX / 32;
    uint2 e[P];
    const int nx = *xn;  // the same for every lane
#pragma unroll
    for (int p = 0; p < P; ++p)
        e[p] = lane + 32 * p < xe ? xl[lane + 32 * p] : make_uint2(0u, 0u);
    const uint2 ex = lane < nx ? xx[lane] : make_uint2(0u, 0u);
    const uint32_t kb = __float_as_uint(*xb) | 0x80000000u;  // ord_key of the bound (>= 0)
    uint32_t bk = 0u, bv = 0xFFFFFFFFu;
#pragma unroll
    for (int p = 0; p < P; ++p) reach_entry<TW>(e[p], lane + 32 * p < xe, tb, bk, bv);
    if (nx > 0) reach_entry<TW>(ex, lane < nx, tb, bk, bv);
    const uint32_t mx = __reduce_max_sync(FULL, bk);
    const uint32_t v = __reduce_min_sync(FULL, bk == mx ? bv : 0xFFFFFFFFu);
    mx_out = mx;  // the lists' best (key 0: none unvisited) for the far list
    v_out = v;
    if (mx <= kb) return -1;  // no unvisited listed node, or one outside may be as good
    return (int)v;
}

// The far list, when the reach list could not decide: the unvisited nodes
// among the row's nearest REACH_FAR (entries REACH_MAX .. of xf: REACH_FAR -
// REACH_MAX ids, two to a 32-bit word) have their choice_info read from the
// row (global memory) and join the lists' best (mx, v); when that beats the
// bound on every node beyond the far list strictly, it is the row's greedy
// choice (ties -> lower id; every node of the largest choice_info is listed),
// else -1.  Three memory round trips: every lane's ids at once, then the
// choice_info of half of them at a time.
template <int TW>
__device__ __forceinline__ int greedy_far(const float *__restrict__ row, const uint16_t *__restrict__ xf,
                                          const float *__restrict__ xfb, const Tabu<TW> &tb, int lane,
                                          uint32_t mx, uint32_t v)
{
    constexpr int W = (REACH_FAR - REACH_MAX) / 64;  // words a lane: 14
    constexpr int H = W / 2;                         // words a half
    const uint32_t *xw = reinterpret_cast<const uint32_t *>(xf);  // 4-byte aligned
    uint32_t w[W];
#pragma unroll
    for (int u = 0; u < W; ++u) w[u] = __ldg(xw + u * 32 + lane);
    uint32_t bk = mx, bv = v;  // the same in every lane
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        uint32_t node[2 * H];
        uint32_t okm = 0;
#pragma unroll
        for (int u = 0; u < H; ++u) {
            node[2 * u] = w[half * H + u] & 0xFFFFu;
            node[2 * u + 1] = w[half * H + u] >> 16;
        }
#pragma unroll
        for (int q = 0; q < 2 * H; ++q) {
            const uint32_t word = tb.word_of((int)node[q]);  // every lane calls it
            okm |= ((word >> (node[q] & 31)) & 1u) ? 0u : (1u << q);
        }
        float x[2 * H];
#pragma unroll
        for (int q = 0; q < 2 * H; ++q) x[q] = ((okm >> q) & 1u) ? __ldcs(row + node[q]) : 0.0f;
#pragma unroll
        for (int q = 0; q < 2 * H; ++q) {
            const uint32_t k = ((okm >> q) & 1u) ? (__float_as_uint(x[q]) | 0x80000000u) : 0u;  // choice_info >= 0
            if (k > bk || (k == bk && k != 0u && node[q] < bv)) {
                bk = k;
                bv = node[q];
            }
        }
    }
    const uint32_t kb = __float_as_uint(*xfb) | 0x80000000u;
    const uint32_t m2 = __reduce_max_sync(FULL, bk);
    if (m2 <= kb) return -1;
    return (int)__reduce_min_sync(FULL, bk == m2 ? bv : 0xFFFFFFFFu);
}

// Bit set in a fallback's result when the whole row was scanned.
constexpr int FB_SCANNED = 1 << 30;

// Candidate-list fallback, out of line so the hot step stays compact:
// fallback = 0 takes the unvisited node of largest choice_info (ties -> lower
// id), first from cur's reach list when that decides it, else from the row;
// fallback = 1 reservoir-samples all unvisited nodes (whole-row stream).  The
// row scans read cur's row with coalesced 16-byte loads, 1024 nodes per round
// trip: on clustered instances most fallbacks come early in the tour, with
// thousands of nodes unvisited, where gathering only the unvisited entries
// costs many more round trips.
// xl / xb / xx / xn: cur's reach list, bound and extra list (xe = 0: none).
template <int TW>
__device__ __noinline__ int cand_fallback(const float *__restrict__ row, int n, const Tabu<TW> tb,
                                          int lane, int mode, uint32_t t, uint32_t ant, uint32_t it,
                                          uint32_t k0, uint32_t k1, uint32_t *err, int cur,
                                          const uint2 *xl, const float *xb, const uint2 *xx,
                                          const int32_t *xn, int xe, const FarList *far)
{
    const bool sparse = TW == 0 && n - (int)t <= SPARSE_SCAN_MAX;  // few nodes left: read only those
    if (mode == 0) {
        if (xe > 0) {
            uint32_t mx, v;
            const int r = greedy_reach<TW>(xl, xb, xe, xx, xn, tb, lane, mx, v);
            if (r >= 0) return r;
            if (TW == 0 && far && !sparse) {
                const FarList f = *far;
                const int r2 = greedy_far<TW>(row, f.xf16 + (size_t)cur * f.fp + REACH_MAX, f.xfb + cur, tb,
                                              lane, mx, v);
                if (r2 >= 0) return r2;
            }
        }
        if (sparse) return scan_unvisited<true>(row, n, tb.w, lane, t, ant, it, k0, k1, err, cur) | FB_SCANNED;
        return scan_row<TW, true, false>(row, n, tb, lane, t, ant, it, k0, k1, err, cur) | FB_SCANNED;
    }
    if (sparse) return scan_unvisited<false>(row, n, tb.w, lane, t, ant, it, k0, k1, err, cur) | FB_SCANNED;
    return scan_row<TW, false, false>(row, n, tb, lane, t, ant, it, k0, k1, err, cur) | FB_SCANNED;
}

// The far list reaches the fallback only from kernels whose tabus live in
// shared memory (TW = 0): far lists exist for n > REACH_FAR_MIN_N > 4096 only,
// and register-tabu kernels pass a constant null (their step loop stays as
// without it).
template <int TW>
__device__ __forceinline__ const FarList *far_of(const ConstructArgs &a)
{
    if constexpr (TW == 0) return a.far;
    else return nullptr;
}
static_assert(REACH_FAR_MIN_N > 4096, "register tabus (n <= 4096) never see a far list");

// Count one fallback step in fbn's low half and, when its row was scanned
// (FB_SCANNED set in the fallback's result), one row scan in its high half;
// return the picked node.
__device__ __forceinline__ int count_fallback(int r, unsigned long long &fbn)
{
    fbn += 1ull + ((unsigned long long)((unsigned)r >> 30) << 32);
    return r & (FB_SCANNED - 1);
}

// Slot `idx` (row cur) of the candidate table: cc / cw are the staged (or
// global) table; PART: only rows below a.stage_rows are staged and the others
// are read from the global table.
template <bool PART>
__device__ __forceinline__ void cand_load(const ConstructArgs &a, const uint16_t *cc, const float *cw,
                                          int cur, int idx, uint32_t &v, float &w)
{
    if constexpr (PART) {
        const bool st = cur < a.stage_rows;
        v = (st ? cc : a.cand16)[idx];
        w = (st ? cw : a.cwinv)[idx];
    } else {
        v = cc[idx];
        w = cw[idx];
    }
}

// One candidate-list step: lane c scores slot c of cur's list.
template <int TW, bool PART>
__device__ __forceinline__ int cand_step(const ConstructArgs &a, const uint16_t *cc,
                                         const float *cw, const Tabu<TW> &tb, int lane,
                                         int cur, float lg, int t, int ant, uint32_t it,
                                         unsigned long long &fbn)
{
    const bool act = lane < a.cl;
    uint32_t v = 0;
    float wi = 0.0f;
    if (act) cand_load<PART>(a, cc, cw, cur, cur * a.cl + lane, v, wi);
    const uint32_t word = tb.word_of((int)v);
    const bool ok = act && !((word >> (v & 31)) & 1u);
    const uint32_t k = ok ? neg_key(__fmul_rn(lg, wi)) : 0u;
    const uint32_t mx = __reduce_max_sync(FULL, k);
    if (__builtin_expect(mx != 0u, 1)) return (int)__reduce_min_sync(FULL, k == mx ? v : 0xFFFFFFFFu);
    return count_fallback(cand_fallback<TW>(a.wmat + (size_t)cur * a.ld, a.n, tb, lane, a.fallback,
                                            (uint32_t)t, (uint32_t)ant, it, a.key0, a.key1, &a.sc->err,
                                            cur, a.xlw + (size_t)cur * a.xe, a.xlb + cur,
                                            a.xxw + (size_t)cur * REACH_EXTRA, a.xxn + cur, a.xe, far_of<TW>(a)),
                          fbn);
}

// Store the window of steps [32w, t_end]: lane l holds entry 32w + l.
__device__ __forceinline__ void store_window(int32_t *trow, int lane, int w, int t_end, int twin)
{
    if (lane <= t_end - 32 * w) trow[32 * w + lane] = twin;
}

// Four steps t = 4g .. 4g+3 with draws lg[0..3]; meanwhile the generator call
// of group g+1 runs in slices and its log2s replace lg.  CHECK: skip t == 0 and
// t >= n and store windows here (first and last groups); otherwise the caller
// stores the window after every eighth group.
template <bool CHECK, int TW, bool PART>
__device__ __forceinline__ void cand_group(const ConstructArgs &a, const uint16_t *cc,
                                           const float *cw, Tabu<TW> &tb, int32_t *trow,
                                           int lane, int ant, uint32_t it, int g, float (&lg)[4],
                                           int &cur, int &twin, unsigned long long &fbn)
{
    uint4 nx = make_uint4((uint32_t)lane, (uint32_t)(g + 1), (uint32_t)ant, it);
    float nl[4];
    const int tb32 = (4 * g) & 31;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (j == 0) philox_rounds_rk<0, 4>(nx, a.rk0, a.rk1);
        if (j == 1) philox_rounds_rk<4, 8>(nx, a.rk0, a.rk1);
        if (j == 2) {
            philox_rounds_rk<8, 10>(nx, a.rk0, a.rk1);
            nl[0] = draw_log2(unit_open(nx.x));
            nl[1] = draw_log2(unit_open(nx.y));
        }
        if (j == 3) {
            nl[2] = draw_log2(unit_open(nx.z));
            nl[3] = draw_log2(unit_open(nx.w));
        }
        const int t = 4 * g + j;
        if (CHECK && (t == 0 || t >= a.n)) continue;
        const int next = cand_step<TW, PART>(a, cc, cw, tb, lane, cur, lg[j], t, ant, it, fbn);
        tb.mark(lane, next);
        twin = (lane == tb32 + j) ? next : twin;
        if (CHECK && ((t & 31) == 31 || t == a.n - 1)) store_window(trow, lane, t >> 5, t, twin);
        cur = next;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) lg[j] = nl[j];
}

// A full group of four steps (t = 4g .. 4g+3, all inside the tour) without a
// branch: a step whose candidates are all visited freezes the rest of the
// group (no mark, no tour entry, cur unchanged), so the four steps and the
// next group's generator work form one straight-line block the compiler can
// interleave.  Only a frozen group leaves the block: that step takes the
// out-of-line fallback and the group's remaining steps run one by one.  The
// result equals cand_group's step for step.
// CL32: cl = 32, every lane holds a candidate.
template <int TW, bool PART, bool CL32>
__device__ __forceinline__ void cand_group_spec(const ConstructArgs &a, const uint16_t *cc,
                                                const float *cw, Tabu<TW> &tb, int lane,
                                                int ant, uint32_t it, int g, float (&lg)[4],
                                                int &cur, int &twin, unsigned long long &fbn)
{
    uint4 nx = make_uint4((uint32_t)lane, (uint32_t)(g + 1), (uint32_t)ant, it);
    float nl[4];
    const int tb32 = (4 * g) & 31;
    const bool act = CL32 || lane < a.cl;
    bool live = true;  // warp-uniform
    int jfail = 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (j == 0) philox_rounds_rk<0, 4>(nx, a.rk0, a.rk1);
        if (j == 1) philox_rounds_rk<4, 8>(nx, a.rk0, a.rk1);
        if (j == 2) {
            philox_rounds_rk<8, 10>(nx, a.rk0, a.rk1);
            nl[0] = draw_log2(unit_open(nx.x));
            nl[1] = draw_log2(unit_open(nx.y));
        }
        if (j == 3) {
            nl[2] = draw_log2(unit_open(nx.z));
            nl[3] = draw_log2(unit_open(nx.w));
        }
        const int idx = CL32 ? cur * 32 + lane : (act ? cur * a.cl + lane : 0);
        uint32_t v;
        float wi;
        cand_load<PART>(a, cc, cw, cur, idx, v, wi);
        const uint32_t word = tb.word_of((int)v);
        const bool ok = act && !((word >> (v & 31)) & 1u);
        const uint32_t k = ok ? neg_key(__fmul_rn(lg[j], wi)) : 0u;
        const uint32_t mx = __reduce_max_sync(FULL, k);
        // (when mx = 0 the step freezes and nxt is not used)
        const uint32_t nxt = __reduce_min_sync(FULL, k == mx ? v : 0xFFFFFFFFu);
        jfail = (live && mx == 0u) ? j : jfail;
        live = live && mx != 0u;
        tb.mark_if(lane, (int)nxt, live);
        twin = (live && lane == tb32 + j) ? (int)nxt : twin;
        cur = live ? (int)nxt : cur;
    }
    if (__builtin_expect(jfail < 4, 0)) {
        // step 4g + jfail: every candidate of cur is visited
        const int t = 4 * g + jfail;
        const int fb = count_fallback(
            cand_fallback<TW>(a.wmat + (size_t)cur * a.ld, a.n, tb, lane, a.fallback, (uint32_t)t,
                              (uint32_t)ant, it, a.key0, a.key1, &a.sc->err, cur,
                              a.xlw + (size_t)cur * a.xe, a.xlb + cur,
                              a.xxw + (size_t)cur * REACH_EXTRA, a.xxn + cur, a.xe, far_of<TW>(a)),
            fbn);
        tb.mark(lane, fb);
        twin = (lane == tb32 + jfail) ? fb : twin;
        cur = fb;
#pragma unroll
        for (int j = 1; j < 4; ++j) {
            if (j <= jfail) continue;
            const int next = cand_step<TW, PART>(a, cc, cw, tb, lane, cur, lg[j], 4 * g + j, ant,
                                                 it, fbn);
            tb.mark(lane, next);
            twin = (lane == tb32 + j) ? next : twin;
            cur = next;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) lg[j] = nl[j];
}

// Whole-row draws of step t for this lane's chunks c = lane + 32u (nodes
// 4c .. 4c+3): the log2 of the four words of Philox(2^31 | c, t, ant, it).
template <int U>
__device__ __forceinline__ void row_draws(int nch, int lane, uint32_t t, uint32_t ant, uint32_t it,
                                          uint32_t k0, uint32_t k1, float (&lg)[U][4])
{
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int c = lane + 32 * u;
        uint4 r = make_uint4(0x80000000u | (uint32_t)(c < nch ? c : 0), t, ant, it);
        philox_rounds<0, 10>(r, k0, k1);
        lg[u][0] = log2f(unit_open(r.x));
        lg[u][1] = log2f(unit_open(r.y));
        lg[u][2] = log2f(unit_open(r.z));
        lg[u][3] = log2f(unit_open(r.w));
    }
}

// Whole-row tour for rows of at most 128 U nodes (one pass of U 16-byte
// chunks per lane): the draws do not depend on the path, so the next step's
// are computed while the current step scans, and the step itself is one
// straight block of U chunk loads, key products and a two-step reduction.
// The same picks as scan_row (ties -> lower id).
template <int U, int TW>
__device__ __forceinline__ void row_tour_pipelined(const ConstructArgs &a, const float *cw, Tabu<TW> &tb,
                                                   int lane, int ant, uint32_t it, int32_t *trow,
                                                   int &cur, int &twin)
{
    const int n = a.n, nch = (n + 3) >> 2;
    float lg[U][4], ln[U][4];
    row_draws<U>(nch, lane, 1u, (uint32_t)ant, it, a.key0, a.key1, lg);
    for (int t = 1; t < n; ++t) {
        const float *row = cw + (size_t)cur * a.ld;
        float4 w4[U];
        uint32_t bits[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = lane + 32 * u;
            const int v0 = c << 2;
            const uint32_t word = tb.word_of(v0 < n ? v0 : n - 1);
            bits[u] = c < nch ? (word >> (v0 & 31)) & 0xFu : 0xFu;
            // generic load: the table may be staged in shared memory
            w4[u] = c < nch ? *reinterpret_cast<const float4 *>(row + v0) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        row_draws<U>(nch, lane, (uint32_t)(t + 1), (uint32_t)ant, it, a.key0, a.key1, ln);
        uint32_t bk = 0u, bv = 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v0 = (lane + 32 * u) << 2;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const bool ok = v0 + e < n && !((bits[u] >> e) & 1u);
                const uint32_t kk = ok ? neg_key(__fmul_rn(lg[u][e], pick_f(w4[u], e))) : 0u;
                if (kk > bk) {  // ascending nodes: ties keep the lower id
                    bk = kk;
                    bv = (uint32_t)(v0 + e);
                }
            }
        }
        const uint32_t mx = __reduce_max_sync(FULL, bk);
        int next = cur;
        if (mx == 0u) {
            if (lane == 0) atomicOr(&a.sc->err, ERR_NO_UNVISITED);
        } else {
            next = (int)__reduce_min_sync(FULL, bk == mx ? bv : 0xFFFFFFFFu);
        }
        tb.mark(lane, next);
        twin = (lane == (t & 31)) ? next : twin;
        if ((t & 31) == 31 || t == n - 1) store_window(trow, lane, t >> 5, t, twin);
        cur = next;
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int e = 0; e < 4; ++e) lg[u][e] = ln[u][e];
    }
}

// Build the tour of ant `ant` (its global index, which keys the draws) into
// trow: a uniform start (Alg. 1), then n - 1 selections.  `it` is the
// iteration index; cc / cw are the candidate table (staged or global) or the
// reciprocal weight matrix (whole-row mode).
template <int MODE, int TW, bool PART = false>
__device__ __forceinline__ void build_tour(const ConstructArgs &a, const uint16_t *cc,
                                           const float *cw, Tabu<TW> &tb, int lane, int ant,
                                           uint32_t it, int32_t *trow)
{
    // Alg. 1: the first node is drawn uniformly
    uint4 s4 = make_uint4(0xFFFFFFFFu, 0u, (uint32_t)ant, it);
    philox_rounds<0, 10>(s4, a.key0, a.key1);
    const int start = (int)(((unsigned long long)s4.x * (unsigned)a.n) >> 32);
    tb.clear(lane);
    tb.mark(lane, start);
    int cur = start;
    int twin = start;  // lane l holds entry 32w + l of the current window
    unsigned long long fbn = 0;

    if constexpr (MODE == CAND) {
        float lg[4];
        {
            uint4 r = make_uint4((uint32_t)lane, 0u, (uint32_t)ant, it);
            philox_rounds<0, 10>(r, a.key0, a.key1);
            lg[0] = 0.0f;  // step 0 is the start node
            lg[1] = draw_log2(unit_open(r.y));
            lg[2] = draw_log2(unit_open(r.z));
            lg[3] = draw_log2(unit_open(r.w));
        }
        cand_group<true, TW, PART>(a, cc, cw, tb, trow, lane, ant, it, 0, lg, cur, twin, fbn);
        int g = 1;
        for (; 4 * g + 3 <= a.n - 1; ++g) {
            if (a.cl == 32)
                cand_group_spec<TW, PART, true>(a, cc, cw, tb, lane, ant, it, g, lg, cur, twin, fbn);
            else
                cand_group_spec<TW, PART, false>(a, cc, cw, tb, lane, ant, it, g, lg, cur, twin, fbn);
            if ((g & 7) == 7) store_window(trow, lane, g >> 3, 4 * g + 3, twin);
        }
        if (4 * g <= a.n - 1)
            cand_group<true, TW, PART>(a, cc, cw, tb, trow, lane, ant, it, g, lg, cur, twin, fbn);
        else if (g > 1 && ((g - 1) & 7) != 7)
            store_window(trow, lane, (g - 1) >> 3, a.n - 1, twin);  // last full group ended it
    } else if (a.n <= 256) {
        row_tour_pipelined<2, TW>(a, cw, tb, lane, ant, it, trow, cur, twin);
    } else if (a.n <= 512) {
        row_tour_pipelined<4, TW>(a, cw, tb, lane, ant, it, trow, cur, twin);
    } else if (a.n <= 1024) {
        row_tour_pipelined<8, TW>(a, cw, tb, lane, ant, it, trow, cur, twin);
    } else {
        for (int t = 1; t < a.n; ++t) {
            const int next = scan_row<TW, false, true>(cw + (size_t)cur * a.ld, a.n, tb, lane,
                                                       (uint32_t)t, (uint32_t)ant, it, a.key0,
                                                       a.key1, &a.sc->err, cur);
            tb.mark(lane, next);
            twin = (lane == (t & 31)) ? next : twin;
            if ((t & 31) == 31 || t == a.n - 1) store_window(trow, lane, t >> 5, t, twin);
            cur = next;
        }
    }
    if (lane == 0 && fbn) {
        atomicAdd(&a.sc->fallback_steps, fbn & 0xFFFFFFFFull);
        if (fbn >> 32) atomicAdd(&a.sc->fallback_scans, fbn >> 32);
    }
}

// Stage `bytes_w` bytes of weights and `bytes_c` of ids into shared memory
// with the bulk-copy engine (thread 0 issues, every thread waits on the
// mbarrier, bounded).  Returns false on a timeout, after which the CTA must
// not use the table.  `parity` is the mbarrier phase this copy completes.
__device__ __forceinline__ bool stage_table(unsigned char *s_w, const void *src_w, uint32_t bytes_w,
                                            unsigned char *s_c, const void *src_c, uint32_t bytes_c,
                                            uint64_t *bar, uint32_t parity, uint32_t *err)
{
    if (threadIdx.x == 0) {
        // the table's shared memory may have been read by this CTA's threads
        // (generic proxy) before the bulk copy (async proxy) overwrites it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, bytes_w + bytes_c);
        const unsigned char *sw = static_cast<const unsigned char *>(src_w);
        for (uint32_t o = 0; o < bytes_w; o += BULK_CHUNK)
            bulk_copy_g2s(s_w + o, sw + o, min(BULK_CHUNK, bytes_w - o), bar);
        const unsigned char *sc = static_cast<const unsigned char *>(src_c);
        for (uint32_t o = 0; o < bytes_c; o += BULK_CHUNK)
            bulk_copy_g2s(s_c + o, sc + o, min(BULK_CHUNK, bytes_c - o), bar);
    }
    if (*reinterpret_cast<volatile uint32_t *>(&g_expire_stage_waits)) {
        const unsigned long long t0 = global_ns();
        while (!*reinterpret_cast<volatile uint32_t *>(&g_never_set) && global_ns() - t0 < EXPIRE_LIMIT_NS) {
        }
        if (threadIdx.x == 0) atomicOr(err, ERR_STAGE_TIMEOUT);
        mbar_wait_bounded(bar, parity, STAGE_LIMIT_NS);  // the copies land before the CTA leaves
        return false;
    }
    if (!mbar_wait_bounded(bar, parity, STAGE_LIMIT_NS)) {
        if (threadIdx.x == 0) atomicOr(err, ERR_STAGE_TIMEOUT);
        // let copies still in flight land before the CTA's memory is released
        mbar_wait_bounded(bar, parity, STAGE_LIMIT_NS);
        return false;
    }
    return true;
}

// STAGED: 0 the table is read from global memory; 1 it is staged whole; 2
// its first a.stage_rows rows are staged (candidate-list mode).  MAXT: threads
// a CTA may have -- 384 (12 warps, registers for the four-step groups) or,
// for tables mostly too large to stage, 512, 768 or 1024 (up to 32 warps with
// fewer registers each: the dependent row reads from L2 are hidden by more
// ants per SM).
template <int MODE, int STAGED, int TW, int MAXT = 384>
__global__ void __launch_bounds__(MAXT, 1) k_construct(const ConstructArgs a, int cons_warps)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t it = (uint32_t)a.iter[0];

    const float *cw = (MODE == CAND) ? a.cwinv : a.wmat;
    const uint16_t *cc = a.cand16;
    size_t off = 0;
    if constexpr (STAGED != 0) {
        unsigned char *s_w = smem;
        off = a.stage_w_bytes;
        unsigned char *s_c = smem + off;
        off += a.stage_c_bytes;
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem + off);
        off += 16;
        if (threadIdx.x == 0) mbar_init(bar, 1);
        __syncthreads();
        if (!stage_table(s_w, cw, a.stage_w_bytes, s_c, a.cand16, a.stage_c_bytes, bar, 0,
                         &a.sc->err))
            return;
        cw = reinterpret_cast<const float *>(s_w);
        cc = reinterpret_cast<const uint16_t *>(s_c);
    }

    Tabu<TW> tb;
    tb.nw = (a.n + 31) >> 5;
    if constexpr (TW == 0) tb.w = reinterpret_cast<uint32_t *>(smem + off) + (size_t)warp * tb.nw;

    const int stride = gridDim.x * cons_warps;
    // `ant` is the global ant index (it keys the draws); this colony's tour rows
    // start at ant_offset, so the row pointer is taken from a base shifted back
    // by ant_offset rows (one induction variable keeps the step loop lean)
    const int ant_end = a.ant_offset + a.m;
    int32_t *const tours_g = a.tours - (size_t)a.ant_offset * a.ld;
    for (int ant = a.ant_offset + blockIdx.x * cons_warps + warp; ant < ant_end; ant += stride)
        build_tour<MODE, TW, STAGED == 2>(a, cc, cw, tb, lane, ant, it, tours_g + (size_t)ant * a.ld);
}

// Candidate lists longer than a warp (32 < cl <= 64): lane l scores slots l
// and l + 32 of the current list (its two draws come from the slots' own
// counters), keeps the better of the two (ties -> lower id) and the warp
// reduces as for one slot a lane.  The table (n x cl x 6 B) is read from L2.
template <int TW>
__device__ __forceinline__ int cand_step2(const ConstructArgs &a, const Tabu<TW> &tb, int lane, int cur,
                                          float lg0, float lg1, int t, int ant, uint32_t it,
                                          unsigned long long &fbn)
{
    const size_t base = (size_t)cur * a.cl;
    const int s1 = lane + 32;
    const bool act1 = s1 < a.cl;
    const uint32_t v0 = a.cand16[base + lane];
    const float w0 = a.cwinv[base + lane];
    const uint32_t v1 = act1 ? a.cand16[base + s1] : v0;
    const float w1 = act1 ? a.cwinv[base + s1] : w0;
    const uint32_t word0 = tb.word_of((int)v0);  // every lane calls both
    const uint32_t word1 = tb.word_of((int)v1);
    const uint32_t k0 = !((word0 >> (v0 & 31)) & 1u) ? neg_key(__fmul_rn(lg0, w0)) : 0u;
    const uint32_t k1 = (act1 && !((word1 >> (v1 & 31)) & 1u)) ? neg_key(__fmul_rn(lg1, w1)) : 0u;
    const bool second = k1 > k0 || (k1 == k0 && k1 != 0u && v1 < v0);
    const uint32_t k = second ? k1 : k0, v = second ? v1 : v0;
    const uint32_t mx = __reduce_max_sync(FULL, k);
    if (__builtin_expect(mx != 0u, 1)) return (int)__reduce_min_sync(FULL, k == mx ? v : 0xFFFFFFFFu);
    return count_fallback(cand_fallback<TW>(a.wmat + (size_t)cur * a.ld, a.n, tb, lane, a.fallback, (uint32_t)t,
                                            (uint32_t)ant, it, a.key0, a.key1, &a.sc->err, cur,
                                            a.xlw + (size_t)cur * a.xe, a.xlb + cur,
                                            a.xxw + (size_t)cur * REACH_EXTRA, a.xxn + cur, a.xe, far_of<TW>(a)),
                          fbn);
}

template <int TW>
__device__ __forceinline__ void build_tour_long(const ConstructArgs &a, Tabu<TW> &tb, int lane, int ant,
                                                uint32_t it, int32_t *trow)
{
    uint4 s4 = make_uint4(0xFFFFFFFFu, 0u, (uint32_t)ant, it);
    philox_rounds<0, 10>(s4, a.key0, a.key1);
    const int start = (int)(((unsigned long long)s4.x * (unsigned)a.n) >> 32);
    tb.clear(lane);
    tb.mark(lane, start);
    int cur = start, twin = start;
    unsigned long long fbn = 0;
    uint4 r0 = make_uint4(0u, 0u, 0u, 0u), r1 = r0;
    for (int t = 1; t < a.n; ++t) {
        if (t == 1 || (t & 3) == 0) {  // the words of slots lane and lane + 32 for group t/4
            r0 = make_uint4((uint32_t)lane, (uint32_t)(t >> 2), (uint32_t)ant, it);
            r1 = make_uint4((uint32_t)(lane + 32), (uint32_t)(t >> 2), (uint32_t)ant, it);
            philox_rounds_rk<0, 10>(r0, a.rk0, a.rk1);
            philox_rounds_rk<0, 10>(r1, a.rk0, a.rk1);
        }
        const float lg0 = draw_log2(unit_open(pick_word(r0, t & 3)));
        const float lg1 = draw_log2(unit_open(pick_word(r1, t & 3)));
        const int next = cand_step2<TW>(a, tb, lane, cur, lg0, lg1, t, ant, it, fbn);
        tb.mark(lane, next);
        twin = (lane == (t & 31)) ? next : twin;
        if ((t & 31) == 31 || t == a.n - 1) store_window(trow, lane, t >> 5, t, twin);
        cur = next;
    }
    if (lane == 0 && fbn) {
        atomicAdd(&a.sc->fallback_steps, fbn & 0xFFFFFFFFull);
        if (fbn >> 32) atomicAdd(&a.sc->fallback_scans, fbn >> 32);
    }
}

// One ant per warp, four warps per CTA, for 32 < cl <= 64.
template <int TW>
__global__ void __launch_bounds__(128) k_construct_long(const ConstructArgs a, int cons_warps)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t it = (uint32_t)a.iter[0];
    Tabu<TW> tb;
    tb.nw = (a.n + 31) >> 5;
    if constexpr (TW == 0) tb.w = reinterpret_cast<uint32_t *>(smem) + (size_t)warp * tb.nw;
    const int stride = gridDim.x * cons_warps;
    const int ant_end = a.ant_offset + a.m;
    int32_t *const tours_g = a.tours - (size_t)a.ant_offset * a.ld;
    for (int ant = a.ant_offset + blockIdx.x * cons_warps + warp; ant < ant_end; ant += stride)
        build_tour_long<TW>(a, tb, lane, ant, it, tours_g + (size_t)ant * a.ld);
}

// Batched construction: one persistent launch builds every ant of
// every colony.  A CTA repeatedly takes the next chunk (one colony, up to one
// ant per warp) from a global counter -- the chunk list is ordered by
// decreasing n so the longest tours start first -- loads that colony's
// arguments, stages its candidate table when table and tabus fit in
// `smem_bytes`, and builds the chunk's tours.  Candidate-list mode only.
template <int TW, int STAGED>
__device__ __forceinline__ void batch_chunk(const ConstructArgs &a, unsigned char *smem,
                                            uint64_t *bar, uint32_t &parity, int first, int count,
                                            int lane, int warp)
{
    const uint32_t it = (uint32_t)a.iter[0];
    const uint16_t *cc = a.cand16;
    const float *cw = a.cwinv;
    size_t off = 0;
    if constexpr (STAGED != 0) {
        const bool ok = stage_table(smem, a.cwinv, a.stage_w_bytes, smem + a.stage_w_bytes, a.cand16,
                                    a.stage_c_bytes, bar, parity, &a.sc->err);
        parity ^= 1u;
        if (!ok) return;
        cw = reinterpret_cast<const float *>(smem);
        cc = reinterpret_cast<const uint16_t *>(smem + a.stage_w_bytes);
        off = (size_t)a.stage_w_bytes + a.stage_c_bytes;
    }
    if (warp >= count) return;
    Tabu<TW> tb;
    tb.nw = (a.n + 31) >> 5;
    if constexpr (TW == 0) tb.w = reinterpret_cast<uint32_t *>(smem + off) + (size_t)warp * tb.nw;
    const int ant = first + warp;  // this colony's ant index (ant_offset = 0)
    build_tour<CAND, TW, STAGED == 2>(a, cc, cw, tb, lane, ant, it, a.tours + (size_t)ant * a.ld);
}

// NARROW: every colony has n <= 2048 (register tabus of 1 or 2 words), which
// lets 16 warps of the tighter code share an SM's registers instead of 12.
template <bool NARROW>
__global__ void __launch_bounds__(NARROW ? 512 : 384, 1)
    k_construct_batch(const ConstructArgs *__restrict__ args, const BatchChunk *__restrict__ chunks,
                      int nchunks, unsigned *counter, uint32_t smem_bytes)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) ConstructArgs s_a;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_chunk, s_mode;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t parity = 0;
    if (threadIdx.x == 0) mbar_init(&s_bar, 1);
    for (;;) {
        __syncthreads();  // the previous chunk is done with s_a and the table
        if (threadIdx.x == 0) s_chunk = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int ci = s_chunk;
        if (ci >= nchunks) break;
        const BatchChunk ch = chunks[ci];
        {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(args + ch.colony);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&s_a);
            for (int i = threadIdx.x; i < (int)(sizeof(ConstructArgs) / 4); i += blockDim.x)
                dst[i] = src[i];
        }
        __syncthreads();
        // stage the whole table when it fits with the tabus, else its first
        // rows (a multiple of 8, at least 64), else none
        if (threadIdx.x == 0) {
            const int tw0 = tabu_words(s_a.n);
            const size_t masks = tw0 ? 0 : (size_t)nwarps * ((s_a.n + 31) >> 5) * sizeof(uint32_t);
            if ((size_t)s_a.stage_w_bytes + s_a.stage_c_bytes + masks <= smem_bytes) {
                s_mode = 1;
                s_a.stage_rows = s_a.n;
            } else {
                const size_t avail = smem_bytes > masks ? smem_bytes - masks : 0;
                const int rows = (int)(avail / ((size_t)s_a.cl * 6)) & ~7;
                s_mode = rows >= 64 && rows < s_a.n ? 2 : 0;
                if (s_mode == 2) {
                    s_a.stage_rows = rows;
                    s_a.stage_w_bytes = (uint32_t)rows * s_a.cl * 4;
                    s_a.stage_c_bytes = (uint32_t)rows * s_a.cl * 2;
                }
            }
        }
        __syncthreads();
        const ConstructArgs &a = s_a;
        const int tw = tabu_words(a.n);
        const int mode = s_mode;
#define MMAS_BATCH_CHUNK(TWV)                                                                   \
    do {                                                                                        \
        if (mode == 1)                                                                          \
            batch_chunk<TWV, 1>(a, smem, &s_bar, parity, ch.first, ch.count, lane, warp);       \
        else if (mode == 2)                                                                     \
            batch_chunk<TWV, 2>(a, smem, &s_bar, parity, ch.first, ch.count, lane, warp);       \
        else                                                                                    \
            batch_chunk<TWV, 0>(a, smem, &s_bar, parity, ch.first, ch.count, lane, warp);       \
    } while (0)
        if (tw == 1) MMAS_BATCH_CHUNK(1);
        else if (NARROW || tw == 2) MMAS_BATCH_CHUNK(2);
        else if (tw == 4) MMAS_BATCH_CHUNK(4);
        else MMAS_BATCH_CHUNK(0);
#undef MMAS_BATCH_CHUNK
    }
}

// ---------------------------------------------------------------------------
// Whole-row variants (Sec. 4.1 compact tabu, Sec. 4.2.1 roulette wheel).
// ---------------------------------------------------------------------------

// Running partial sums q[0..3] of lane l's four positions 128r + 4l .. +3 of
// round r, x() giving each position's weight (0 beyond N), plus the weights.
template <class X>
__device__ __forceinline__ void rwm_lane(X x, int r, int lane, int N, float (&w)[4], float (&q)[4])
{
    const int p0 = 128 * r + 4 * lane;
    x(p0, N, w);
    q[0] = w[0];
    q[1] = __fadd_rn(q[0], w[1]);
    q[2] = __fadd_rn(q[1], w[2]);
    q[3] = __fadd_rn(q[2], w[3]);
}

// Inclusive lane scan, S_l <- S_l + S_{l-d} for d = 1, 2, 4, 8, 16.
__device__ __forceinline__ float rwm_scan(float S, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float v = __shfl_up_sync(FULL, S, d);
        if (lane >= d) S = __fadd_rn(S, v);
    }
    return S;
}

// The same procedure for N <= 128 RC: the first pass keeps each round's
// weights, partial sums and lane scan in registers, so the search pass reuses
// them instead of reloading and rescanning (the same operations, the same pick).
template <int RC, class X>
__device__ __forceinline__ int rwm_pick_cached(X x, int N, float u, int lane)
{
    const int rounds = (N + 127) >> 7;
    float w[RC][4], q[RC][4], S[RC], P[RC];
    float total = 0.0f;
#pragma unroll
    for (int r = 0; r < RC; ++r) {
        if (r < rounds) {
            rwm_lane(x, r, lane, N, w[r], q[r]);
            S[r] = rwm_scan(q[r][3], lane);
            P[r] = __shfl_up_sync(FULL, S[r], 1);
            if (lane == 0) P[r] = 0.0f;
            total = __fadd_rn(total, __shfl_sync(FULL, S[r], 31));
        }
    }
    const float theta = __fmul_rn(u, total);
    float off = 0.0f;
    int last = -1;
#pragma unroll
    for (int r = 0; r < RC; ++r) {
        if (r < rounds) {
            const float base = __fadd_rn(off, P[r]);
            int hit = 4;
#pragma unroll
            for (int e = 3; e >= 0; --e) {
                const int p = 128 * r + 4 * lane + e;
                if (p < N && w[r][e] > 0.0f) {
                    last = p > last ? p : last;
                    if (__fadd_rn(base, q[r][e]) > theta) hit = e;
                }
            }
            const unsigned b = __ballot_sync(FULL, hit < 4);
            if (b) {
                const int wl = __ffs(b) - 1;
                return 128 * r + 4 * wl + __shfl_sync(FULL, hit, wl);
            }
            off = __fadd_rn(off, __shfl_sync(FULL, S[r], 31));
        }
    }
    return (int)__reduce_max_sync(FULL, (unsigned)(last + 1)) - 1;
}

// The parallel roulette wheel over positions [0, N) with draw u: the exact
// single-precision procedure (rounds of 128 positions, lane partial sums,
// lane scan, running round offset; first position whose cumulative sum
// exceeds u * total, else the last positive one).  Every lane returns it;
// -1 when no weight is positive.
template <class X>
__device__ __forceinline__ int rwm_pick(X x, int N, float u, int lane)
{
    const int rounds = (N + 127) >> 7;
    float total = 0.0f;
    for (int r = 0; r < rounds; ++r) {
        float w[4], q[4];
        rwm_lane(x, r, lane, N, w, q);
        total = __fadd_rn(total, __shfl_sync(FULL, rwm_scan(q[3], lane), 31));
    }
    const float theta = __fmul_rn(u, total);
    float off = 0.0f;
    int last = -1;
    for (int r = 0; r < rounds; ++r) {
        float w[4], q[4];
        rwm_lane(x, r, lane, N, w, q);
        const float S = rwm_scan(q[3], lane);
        float prev = __shfl_up_sync(FULL, S, 1);
        if (lane == 0) prev = 0.0f;
        const float base = __fadd_rn(off, prev);
        int hit = 4;
#pragma unroll
        for (int e = 3; e >= 0; --e) {
            const int p = 128 * r + 4 * lane + e;
            if (p < N && w[e] > 0.0f) {
                last = p > last ? p : last;
                if (__fadd_rn(base, q[e]) > theta) hit = e;
            }
        }
        const unsigned b = __ballot_sync(FULL, hit < 4);
        if (b) {
            const int wl = __ffs(b) - 1;
            return 128 * r + 4 * wl + __shfl_sync(FULL, hit, wl);
        }
        off = __fadd_rn(off, __shfl_sync(FULL, S, 31));
    }
    return (int)__reduce_max_sync(FULL, (unsigned)(last + 1)) - 1;
}

// One warp's compact list of unvisited nodes (shared memory, 16-bit ids).
struct Compact {
    uint16_t *e;
    int L, n;
    __device__ __forceinline__ void init(int lane)
    {
        for (int j = lane; j < n; j += 32) e[j] = (uint16_t)j;
        L = n;
        __syncwarp();
    }
    // remove the node at slot j (Sec. 4.1): the last node takes its place
    __device__ __forceinline__ void remove(int j, int lane)
    {
        if (lane == 0) {
            if (j == L - 1) {
                e[j] = (uint16_t)n;
            } else {
                const int last = e[L - 1];
                e[j] = (uint16_t)last;
                e[last] = (uint16_t)j;
            }
        }
        --L;
        __syncwarp();
    }
};

// One whole-row tour under the variant (SEL: 0 reservoir sampling, 1
// roulette wheel; CT: compact list, else the bitmask tabu tb).  `row0` is the
// weight matrix: 1/choice_info for reservoir sampling, choice_info for the
// roulette wheel.
template <int SEL, bool CT, int TW>
__device__ __forceinline__ void build_tour_var(const ConstructArgs &a, const float *row0, Tabu<TW> &tb,
                                               Compact &cl, int lane, int ant, uint32_t it, int32_t *trow)
{
    uint4 s4 = make_uint4(0xFFFFFFFFu, 0u, (uint32_t)ant, it);
    philox_rounds<0, 10>(s4, a.key0, a.key1);
    const int start = (int)(((unsigned long long)s4.x * (unsigned)a.n) >> 32);
    int cur = start, slot = start, twin = start;
    if constexpr (CT) {
        cl.init(lane);
    } else {
        tb.clear(lane);
        tb.mark(lane, start);
    }
    for (int t = 1; t < a.n; ++t) {
        if constexpr (CT) cl.remove(slot, lane);
        const float *row = row0 + (size_t)cur * a.ld;
        int next = -1, nslot = -1;
        if constexpr (SEL == 1) {
            uint4 r4 = make_uint4(0xFFFFFFFEu, (uint32_t)t, (uint32_t)ant, it);
            philox_rounds<0, 10>(r4, a.key0, a.key1);
            const float u = unit_open(r4.x);
            if constexpr (CT) {
                const uint16_t *e = cl.e;
                auto x = [&](int p0, int N, float (&w)[4]) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) w[k] = p0 + k < N ? row[e[p0 + k]] : 0.0f;
                };
                nslot = cl.L <= 256 ? rwm_pick_cached<2>(x, cl.L, u, lane) : rwm_pick(x, cl.L, u, lane);
                next = nslot >= 0 ? (int)cl.e[nslot] : -1;
            } else {
                auto x = [&](int p0, int N, float (&w)[4]) {
                    const uint32_t bits = (tb.word_of(p0 < N ? p0 : 0) >> (p0 & 31)) & 0xFu;
                    const float4 v = p0 < N ? *reinterpret_cast<const float4 *>(row + p0)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
                    w[0] = p0 < N && !(bits & 1u) ? v.x : 0.0f;
                    w[1] = p0 + 1 < N && !(bits & 2u) ? v.y : 0.0f;
                    w[2] = p0 + 2 < N && !(bits & 4u) ? v.z : 0.0f;
                    w[3] = p0 + 3 < N && !(bits & 8u) ? v.w : 0.0f;
                };
                next = a.n <= 256 ? rwm_pick_cached<2>(x, a.n, u, lane) : rwm_pick(x, a.n, u, lane);
            }
        } else {
            // reservoir sampling over the compact list, slot-keyed draws
            uint32_t bk = 0, bv = 0xFFFFFFFFu, bs = 0;
            for (int r = 0; 128 * r < cl.L; ++r) {
                const int j0 = 128 * r + 4 * lane;
                if (j0 >= cl.L) continue;
                uint4 d4 = make_uint4(0x40000000u | (uint32_t)(32 * r + lane), (uint32_t)t, (uint32_t)ant, it);
                philox_rounds<0, 10>(d4, a.key0, a.key1);
                const uint32_t wd[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int j = j0 + k;
                    if (j >= cl.L) break;
                    const uint32_t v = cl.e[j];
                    const uint32_t kk = ord_key(__fmul_rn(log2f(unit_open(wd[k])), row[v]));
                    if (kk > bk || (kk == bk && v < bv)) {
                        bk = kk;
                        bv = v;
                        bs = (uint32_t)j;
                    }
                }
            }
            const uint32_t mx = __reduce_max_sync(FULL, bk);
            const uint32_t win = __reduce_min_sync(FULL, bk == mx ? bv : 0xFFFFFFFFu);
            const unsigned owner = __ballot_sync(FULL, bv == win && bk == mx);
            next = mx ? (int)win : -1;
            nslot = owner ? (int)__shfl_sync(FULL, bs, __ffs(owner) - 1) : -1;
        }
        if (next < 0) {  // no positive weight: cannot happen with tau_min > 0
            if (lane == 0) atomicOr(&a.sc->err, ERR_NO_UNVISITED);
            return;
        }
        if constexpr (!CT) tb.mark(lane, next);
        twin = (lane == (t & 31)) ? next : twin;
        if ((t & 31) == 31 || t == a.n - 1) store_window(trow, lane, t >> 5, t, twin);
        cur = next;
        slot = nslot;
    }
}

template <int SEL, bool CT, bool STAGED, int TW>
__global__ void __launch_bounds__(384, 1) k_construct_var(const ConstructArgs a, int cons_warps)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t it = (uint32_t)a.iter[0];
    const float *row0 = a.wmat;
    size_t off = 0;
    if constexpr (STAGED) {
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem + a.stage_w_bytes);
        if (threadIdx.x == 0) mbar_init(bar, 1);
        __syncthreads();
        if (!stage_table(smem, a.wmat, a.stage_w_bytes, nullptr, nullptr, 0, bar, 0, &a.sc->err)) return;
        row0 = reinterpret_cast<const float *>(smem);
        off = (size_t)a.stage_w_bytes + 16;
    }
    Tabu<TW> tb;
    tb.nw = (a.n + 31) >> 5;
    Compact cl;
    cl.n = a.n;
    cl.L = a.n;
    cl.e = nullptr;
    if constexpr (CT) {
        const size_t per = ((size_t)a.n * 2 + 15) & ~size_t(15);
        cl.e = reinterpret_cast<uint16_t *>(smem + off + (size_t)warp * per);
    } else {
        if constexpr (TW == 0) tb.w = reinterpret_cast<uint32_t *>(smem + off) + (size_t)warp * tb.nw;
    }
    const int stride = gridDim.x * cons_warps;
    const int ant_end = a.ant_offset + a.m;
    int32_t *const tours_g = a.tours - (size_t)a.ant_offset * a.ld;
    for (int ant = a.ant_offset + blockIdx.x * cons_warps + warp; ant < ant_end; ant += stride)
        build_tour_var<SEL, CT, TW>(a, row0, tb, cl, lane, ant, it, tours_g + (size_t)ant * a.ld);
}

using KernelFn = void (*)(const ConstructArgs, int);

// tw: tabu words per lane (1, 2, 4), or 0 for the shared-memory tabu
// staged: 0 none, 1 the whole table, 2 its first rows (candidate lists only)
KernelFn pick_kernel(int mode, int staged, int tw)
{
    static const KernelFn cand[3][4] = {
        {k_construct<CAND, 0, 0>, k_construct<CAND, 0, 1>, k_construct<CAND, 0, 2>, k_construct<CAND, 0, 4>},
        {k_construct<CAND, 1, 0>, k_construct<CAND, 1, 1>, k_construct<CAND, 1, 2>, k_construct<CAND, 1, 4>},
        {k_construct<CAND, 2, 0>, k_construct<CAND, 2, 1>, k_construct<CAND, 2, 2>, k_construct<CAND, 2, 4>},
    };
    static const KernelFn rowk[2][4] = {
        {k_construct<ROW, 0, 0>, k_construct<ROW, 0, 1>, k_construct<ROW, 0, 2>, k_construct<ROW, 0, 4>},
        {k_construct<ROW, 1, 0>, k_construct<ROW, 1, 1>, k_construct<ROW, 1, 2>, k_construct<ROW, 1, 4>},
    };
    const int ti = tw == 4 ? 3 : tw;  // 0, 1, 2, 4 -> 0, 1, 2, 3
    return mode == CAND ? cand[staged][ti] : rowk[staged ? 1 : 0][ti];
}

// the 32-warp form, tabus in shared memory, rows read through L1 and L2
// The smallest of the 512-, 768- and 1024-thread builds that holds `warps`
// warps (fewer threads a CTA leave more registers a thread).
KernelFn pick_kernel_wide(int warps)
{
    return warps <= 16 ? k_construct<CAND, 0, 0, 512>
                       : (warps <= 24 ? k_construct<CAND, 0, 0, 768> : k_construct<CAND, 0, 0, 1024>);
}

KernelFn pick_kernel_long(int tw)
{
    return tw == 1 ? k_construct_long<1>
                   : (tw == 2 ? k_construct_long<2> : (tw == 4 ? k_construct_long<4> : k_construct_long<0>));
}

// whole-row variants: (sel, ct) != (0, 0); TW 1 (n <= 1024) or 0 for the bitmask
KernelFn pick_kernel_var(int sel, int ct, int staged, int tw)
{
    if (ct) {
        if (sel) return staged ? k_construct_var<1, true, true, 1> : k_construct_var<1, true, false, 1>;
        return staged ? k_construct_var<0, true, true, 1> : k_construct_var<0, true, false, 1>;
    }
    if (tw == 1) return staged ? k_construct_var<1, false, true, 1> : k_construct_var<1, false, false, 1>;
    return staged ? k_construct_var<1, false, true, 0> : k_construct_var<1, false, false, 0>;
}

}  // namespace

cudaError_t set_stage_wait_expiry(bool on)
{
    const uint32_t v = on ? 1u : 0u;
    return cudaMemcpyToSymbol(g_expire_stage_waits, &v, sizeof(v));
}

cudaError_t plan_construct(const ConstructArgs &a, int num_sms, size_t smem_optin,
                           ConstructPlan *plan)
{
    const bool row = a.cl == 0;
    const bool var = row && (a.sel != 0 || a.ct != 0);
    const int nw = (a.n + 31) / 32;
    plan->tw = var ? (a.n <= 1024 ? 1 : 0) : tabu_words(a.n);
    plan->longl = !row && a.cl > 32;
    if (plan->longl) {  // 32 < cl <= 64: two slots a lane, rows from L2
        plan->wide = 0;
        plan->staged = 0;
        plan->stage_rows = 0;
        plan->cons_warps = 4;
        plan->gen_warps = 0;
        plan->grid = (a.m + 3) / 4;
        plan->smem = plan->tw ? 0 : (size_t)4 * nw * sizeof(uint32_t);
        return cudaFuncSetAttribute(reinterpret_cast<const void *>(pick_kernel_long(plan->tw)),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan->smem);
    }
    // most rows of the candidate table unstageable (under a quarter of it fits
    // beside the tabus of 12 warps): 32 warps per CTA (MAXT = 1024), the rows
    // read through L1 and L2
    plan->wide = 0;
    if (!row && !var && plan->tw == 0) {
        const size_t tabus12 = (size_t)12 * nw * sizeof(uint32_t);
        const size_t room = smem_optin > 16 + tabus12 ? smem_optin - 16 - tabus12 : 0;
        plan->wide = room / ((size_t)a.cl * 6) * 4 < (size_t)a.n && a.m > 12 * num_sms;
    }
    const int max_warps = plan->wide ? 32 : 12;
    // per-warp shared memory besides the table: the compact list, or the tabu
    // bitmask when it does not live in registers
    const size_t per_warp = (var && a.ct) ? (((size_t)a.n * 2 + 15) & ~size_t(15))
                                          : (plan->tw ? 0 : (size_t)nw * sizeof(uint32_t));
    const size_t table = row ? (size_t)a.n * a.ld * sizeof(float)
                             : (size_t)a.stage_w_bytes + a.stage_c_bytes;
    // staged: one CTA per SM (the table fills its shared memory) carrying
    // ceil(m / #SMs) ants, at most max_warps warps; warps loop over further ants
    int w = (a.m + num_sms - 1) / num_sms;
    w = w < 1 ? 1 : (w > max_warps ? max_warps : w);
    const size_t masks = (size_t)w * per_warp;
    const size_t need = table + 16 + masks;
    // candidate lists too large to stage whole: stage their first rows (a
    // multiple of 8), the rest is read from global memory
    const size_t avail = smem_optin > 16 + masks ? smem_optin - 16 - masks : 0;
    const int part_rows = row ? 0 : (int)(avail / ((size_t)a.cl * 6)) & ~7;
    plan->stage_rows = a.n;
    const int wave = w;  // ants a CTA builds at once
    if (plan->wide) {
        // no staging: shared memory holds only the tabus, which leaves L1 room
        // to cache the candidate rows (measured faster than staging the few
        // rows that fit: 84 -> 69 ms at n = 18,500).  The ants run in rounds of
        // one per warp; the fewest rounds that 32 warps a CTA need are filled
        // evenly, so the last round is not a nearly idle one (n = m = 10,000:
        // 22 warps, 3 full rounds, 22.6 -> 18.4 ms)
        const int per_round = num_sms * 32;
        const int rounds = (a.m + per_round - 1) / per_round;
        w = (a.m + num_sms * rounds - 1) / (num_sms * rounds);
        plan->staged = 0;
        plan->cons_warps = w;
        plan->gen_warps = 0;
        const int g = (a.m + w - 1) / w;
        plan->grid = g < num_sms ? g : num_sms;
        plan->smem = (size_t)w * per_warp;
    } else if (need <= smem_optin && table < (1u << 30)) {
        plan->staged = 1;
        plan->cons_warps = w;
        plan->gen_warps = 0;
        const int g = (a.m + wave - 1) / wave;
        plan->grid = g < num_sms ? g : num_sms;
        plan->smem = need;
    } else if (!var && part_rows >= 64 && part_rows < a.n) {
        plan->staged = 2;
        plan->stage_rows = part_rows;
        plan->cons_warps = w;
        plan->gen_warps = 0;
        const int g = (a.m + wave - 1) / wave;
        plan->grid = g < num_sms ? g : num_sms;
        plan->smem = (size_t)part_rows * a.cl * 6 + 16 + masks;
    } else {
        plan->staged = 0;
        plan->cons_warps = 4;
        plan->gen_warps = 0;
        plan->grid = (a.m + 3) / 4;
        plan->smem = (size_t)4 * per_warp;
    }
    KernelFn k = var ? pick_kernel_var(a.sel, a.ct, plan->staged, plan->tw)
                     : (plan->wide ? pick_kernel_wide(plan->cons_warps)
                                   : pick_kernel(row ? ROW : CAND, plan->staged, plan->tw));
    return cudaFuncSetAttribute(reinterpret_cast<const void *>(k),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan->smem);
}

cudaError_t prepare_construct_batch(size_t smem_bytes, bool narrow)
{
    const void *k = narrow ? reinterpret_cast<const void *>(k_construct_batch<true>)
                           : reinterpret_cast<const void *>(k_construct_batch<false>);
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

cudaError_t launch_construct_batch(const ConstructArgs *args, const BatchChunk *chunks, int nchunks,
                                   unsigned *counter, int grid, int warps, size_t smem_bytes,
                                   bool narrow, cudaStream_t s)
{
    if (narrow)
        k_construct_batch<true><<<grid, warps * 32, smem_bytes, s>>>(args, chunks, nchunks, counter,
                                                                     (uint32_t)smem_bytes);
    else
        k_construct_batch<false><<<grid, warps * 32, smem_bytes, s>>>(args, chunks, nchunks, counter,
                                                                      (uint32_t)smem_bytes);
    return cudaGetLastError();
}

cudaError_t launch_construct(const ConstructArgs &a, const ConstructPlan &plan, cudaStream_t s)
{
    ConstructArgs b = a;
    b.stage_rows = plan.stage_rows;
    if (!plan.staged) {
        b.stage_w_bytes = 0;
        b.stage_c_bytes = 0;
    } else if (plan.staged == 2) {
        b.stage_w_bytes = (uint32_t)plan.stage_rows * a.cl * 4;
        b.stage_c_bytes = (uint32_t)plan.stage_rows * a.cl * 2;
    } else if (a.cl == 0) {
        b.stage_w_bytes = (uint32_t)((size_t)a.n * a.ld * sizeof(float));
        b.stage_c_bytes = 0;
    }
    const bool var = a.cl == 0 && (a.sel != 0 || a.ct != 0);
    KernelFn k = var ? pick_kernel_var(a.sel, a.ct, plan.staged, plan.tw)
                     : plan.longl ? pick_kernel_long(plan.tw)
                     : (plan.wide ? pick_kernel_wide(plan.cons_warps)
                                  : pick_kernel(a.cl == 0 ? ROW : CAND, plan.staged, plan.tw));
    k<<<plan.grid, (plan.cons_warps + plan.gen_warps) * 32, plan.smem, s>>>(b, plan.cons_warps);
    return cudaGetLastError();
}

}  // namespace mmas
