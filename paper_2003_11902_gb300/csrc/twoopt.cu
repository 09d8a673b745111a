// 2-opt local search (Sec. 5.7): Bentley's neighbour-list 2-opt with
// don't-look bits, first improvement, on whole tours.
//
// One CTA improves one tour held in shared memory (tour and position of each
// city, the length of each tour edge, don't-look bits: 13 bytes per city).
// The sequential search visits the cities in index order, skipping those
// whose don't-look bit is set; a city without a move gets its bit set, a move
// clears the bits of its four cities and the visit continues after the moving
// city; a run ends after a pass with no move, and runs (from cleared bits)
// repeat until a run makes no move.
//
// Here each round evaluates a window of consecutive cities in parallel, one
// warp per city -- or, with neighbour lists of at most 16, one half-warp per
// city (lane h examines neighbour h on both sides, and ballots pick the first
// improving neighbour in list order) -- against the current tour, and applies
// the lowest-index improving move; the window's earlier cities had no move, so
// they get their bits set.  That is exactly the sequential search, move for
// move, for any window size: the window is one city a searching group (at most
// 16) after a move (moves come densely, so a small window wastes few
// evaluations) and doubles, up to blockDim, while windows find none.
//
// Round protocol.  A searching group with a move records it in its own slot
// (city, side, the two positions, the two new edge lengths) and publishes its
// city by atomic minimum, so the lowest city wins; the winner's slot then
// describes the whole move.  The minima live in three rotating words: after the round's
// barrier a word two rounds ahead is reset, which no thread can still be
// reading, so a round without a move costs one barrier.
// A move costs one more: warp 0 alone applies it -- bits of the skipped
// cities, the reversal of the shorter path (18 cities on average on the
// clustered n = 3800 workload), the two new edges, the four cleared bits --
// while the other warps wait at the barrier.
//
// Several moves a round.  A search reads the tour only at the positions of
// its city and of its neighbours, and one step either side of them (its
// footprint).  A move rewrites positions pa - 1 .. pb + 1 only (the reversed
// path [pa..pb] and the two edges that border it).  So a search whose
// footprint lies outside pa - 2 .. pb + 2 returns the same result on the new
// tour as on the old one.  The window's first cities (one a group) keep their
// footprints; after the search one warp per kept city tests its footprint against
// the ranges of the moves of the earlier kept cities (computed from their
// move records, which stay exact for every move that is applied), and warp 0
// walks on from the round's first move: a city whose footprint misses every
// move applied so far keeps its result -- no move: its bit is set; a move: it
// is applied next; a city skipped for its bit: its bit stays set -- and the
// walk stops at the first city it cannot vouch for, where the next round
// starts.  That is again the sequential search move for move; on the
// clustered n = 3800 workload it takes about a third of the rounds.
//
// Neighbour lists are the colony's candidate lists.  For the iteration-best
// tour (one CTA) the coordinates and 16-bit lists are staged in shared memory
// when they fit, so a neighbour costs shared loads only; otherwise neighbour
// distances come from a table precomputed at set-up.  Distances are the exact
// integer ones (coordinates or the explicit matrix).
#include <climits>

#include "distance.cuh"
#include "internal.cuh"
#include "twoopt.cuh"

namespace mmas {

namespace {

// Testing aid (mmas_debug_two_opt_move_cap): when positive, replaces the move
// cap of 64 n, so a test can make a search hit it.
__device__ long long g_two_opt_cap;


// Shared-memory layout (byte offsets), identical on host and device.
struct Layout {
    uint32_t xy, nn, edge, tour, pos, dlb, total;
    __host__ __device__ static Layout make(int n, int k, bool staged)
    {
        Layout L;
        uint32_t off = 0;
        L.xy = off;
        if (staged) off += 8u * n;
        off = (off + 15u) & ~15u;
        L.nn = off;
        if (staged) off += 2u * n * k;
        off = (off + 15u) & ~15u;
        L.edge = off;
        off += 4u * n;
        L.tour = off;
        off += 4u * n;
        L.pos = off;
        off += 4u * n;
        L.dlb = off;  // don't-look bits, one per city
        off += 4u * ((n + 31u) / 32u);
        L.total = off + 16u;
        return L;
    }
};

// The tour image: tour[i], pos[c], edge[i] = d(tour[i], tour[i+1 mod n]).
struct TourView {
    int32_t *tour, *pos, *edge;
    int n;
    __device__ __forceinline__ int nxt(int i) const { return i + 1 == n ? 0 : i + 1; }
    __device__ __forceinline__ int prv(int i) const { return i == 0 ? n - 1 : i - 1; }
};

// Distances and neighbour lists, from shared memory when staged.
template <bool XY, bool STAGED>
struct Geometry {
    const TwoOptArgs &a;
    const int2 *sxy;
    const uint16_t *snn;
    __device__ __forceinline__ int d(int u, int v) const
    {
        if constexpr (STAGED)
            return euc2d_exact(sxy[u], sxy[v]);
        else if constexpr (XY)
            return euc2d_exact(__ldg(a.xy + u), __ldg(a.xy + v));
        else
            return __ldg(a.dist + (size_t)u * a.ld + v);
    }
    __device__ __forceinline__ int neighbour(int c, int h) const
    {
        if constexpr (STAGED)
            return snn[c * a.k + h];
        else
            return __ldg(a.nn + (size_t)c * a.k + h);
    }
    // squared Euclidean distance (coordinate instances)
    __device__ __forceinline__ long long sq(int u, int v) const
    {
        int2 pu, pv;
        if constexpr (STAGED) {
            pu = sxy[u];
            pv = sxy[v];
        } else {
            pu = __ldg(a.xy + u);
            pv = __ldg(a.xy + v);
        }
        const long long dx = (long long)pu.x - pv.x, dy = (long long)pu.y - pv.y;
        return dx * dx + dy * dy;
    }
    // d(c, c2) for c2, neighbour h of c
    __device__ __forceinline__ int neighbour_dist(int c, int h, int c2) const
    {
        if constexpr (STAGED)
            return euc2d_exact(sxy[c], sxy[c2]);
        else
            return __ldg(a.nnd + (size_t)c * a.k + h);
    }
};

// A move at city c1.  side 0 = successor side (remove c1->succ(c1) and
// c2->succ(c2), add c1-c2 and succ(c1)-succ(c2)); side 1 = predecessor side
// (remove pred(c1)->c1 and pred(c2)->c2, add c1-c2 and pred(c1)-pred(c2));
// p = pos[c1], q = pos[c2]; d12 = d(c1, c2) and d34 the other added edge.
struct Move {
    int32_t c1, side, p, q, d12, d34;
};

// nint(sqrt(s)) < t, exactly, from the squared distance s: for t >= 1 it holds
// iff sqrt(s) < t - 1/2 (sqrt(s) is never a half-integer), that is s <= t^2 - t.
__device__ __forceinline__ bool nint_sqrt_below(long long s, long long t)
{
    return t > 0 && s <= t * t - t;
}

// First improving move at city c1, searched by one warp (PAIR: by one half of
// a warp, lanes 16 half .. 16 half + 15, each half with its own city; k <= 16):
// lane h examines neighbour h (h < k) on both sides.  The sequential scan of a
// side stops at the first neighbour not closer than the tour neighbour on that
// side; the lists are sorted by distance, so the neighbours it examines are
// exactly those with d(c1, c2) below that radius, and its first improving one
// is the lowest such lane whose gain is positive.  The successor side wins
// over the predecessor side.  Every lane of the warp (the half) returns the
// same result; act = false: a half with nothing to search (c1 must still be a
// city), which finds nothing.  Every lane of the warp calls it.
// fp (when not null) receives the footprint's positions: p = pos[c1] in
// fp[0], and pos of neighbour h in fp[1 + h].
template <bool XY, bool STAGED, bool PAIR>
__device__ __forceinline__ bool find_move_warp(const TwoOptArgs &a, const Geometry<XY, STAGED> &g,
                                               const TourView &tv, int c1, int lane, bool act,
                                               Move &mv, uint16_t *fp)
{
    const int hl = PAIR ? (lane & 15) : lane;  // lane within the searching group
    const int sh = PAIR ? (lane & 16) : 0;     // the group's first lane
    const int p = tv.pos[c1];
    if (fp && hl == 0) fp[0] = (uint16_t)p;
    const int pn = tv.nxt(p), pp = tv.prv(p);
    const int s1 = tv.tour[pn], p1 = tv.tour[pp];
    const int rs = tv.edge[p], rp = tv.edge[pp];
    bool vs = false, vp = false;
    int q = 0, d12 = 0, tn = 0, tp = 0, dss = 0, dpp = 0;
    if (act && hl < a.k) {
        const int c2 = g.neighbour(c1, hl);
        d12 = g.neighbour_dist(c1, hl, c2);
        q = tv.pos[c2];
        if (fp) fp[1 + hl] = (uint16_t)q;
        const int qn = tv.nxt(q), qp = tv.prv(q);
        tn = tv.tour[qn];
        tp = tv.tour[qp];
        // improving: d(s1, succ c2) < rs + d(c2, succ c2) - d12, and alike on
        // the predecessor side; with coordinates the test runs on the squared
        // distance, without a square root
        const long long ts = (long long)rs + tv.edge[q] - d12, tq = (long long)rp + tv.edge[qp] - d12;
        if constexpr (XY) {
            vs = d12 < rs && nint_sqrt_below(g.sq(s1, tn), ts);
            vp = d12 < rp && nint_sqrt_below(g.sq(p1, tp), tq);
        } else {
            dss = g.d(s1, tn);
            dpp = g.d(p1, tp);
            vs = d12 < rs && dss < ts;
            vp = d12 < rp && dpp < tq;
        }
    }
    unsigned ms = __ballot_sync(0xFFFFFFFFu, vs), mp = __ballot_sync(0xFFFFFFFFu, vp);
    if constexpr (PAIR) {
        ms = (ms >> sh) & 0xFFFFu;
        mp = (mp >> sh) & 0xFFFFu;
    } else {
        if ((ms | mp) == 0u) return false;  // the same in every lane
    }
    const bool found = (ms | mp) != 0u;
    const int h = found ? __ffs(ms ? ms : mp) - 1 : 0;
    int d34 = ms ? dss : dpp;
    if constexpr (XY) {
        if (found && hl == h) d34 = ms ? g.d(s1, tn) : g.d(p1, tp);  // the added edge, exactly
    }
    mv.c1 = c1;
    mv.side = ms ? 0 : 1;
    mv.p = p;
    mv.q = __shfl_sync(0xFFFFFFFFu, q, sh + h);
    mv.d12 = __shfl_sync(0xFFFFFFFFu, d12, sh + h);
    mv.d34 = __shfl_sync(0xFFFFFFFFu, d34, sh + h);
    return found;
}

// Reverse tour[pa..pb] (len cities, cyclic) with `count` threads numbered
// `t`; the len - 1 edges inside the path reverse with it.
__device__ __forceinline__ void reverse_path(const TourView &tv, int pa, int pb, int len, int t,
                                             int count)
{
    const int n = tv.n;
    for (int s2 = t; s2 < len / 2; s2 += count) {
        int i = pa + s2, j = pb - s2;
        if (i >= n) i -= n;
        if (j < 0) j += n;
        const int ci = tv.tour[i], cj = tv.tour[j];
        tv.tour[i] = cj;
        tv.pos[cj] = i;
        tv.tour[j] = ci;
        tv.pos[ci] = j;
    }
    for (int s2 = t; s2 < (len - 1) / 2; s2 += count) {
        int i = pa + s2, j = pb - 1 - s2;
        if (i >= n) i -= n;
        if (j < 0) j += n;
        const int ei = tv.edge[i];
        tv.edge[i] = tv.edge[j];
        tv.edge[j] = ei;
    }
}

// Don't-look bits: bit c & 31 of word c >> 5.
__device__ __forceinline__ bool dlb_get(const uint32_t *dlb, int c) { return (dlb[c >> 5] >> (c & 31)) & 1u; }

// Set the bits of cities [lo, hi); thread t of `count` takes words t, t + count,
// ... of the range, so no word has two writers.
__device__ __forceinline__ void dlb_set_range(uint32_t *dlb, int lo, int hi, int t, int count)
{
    if (hi <= lo) return;
    const int q0 = lo >> 5, q1 = (hi - 1) >> 5;
    for (int q = q0 + t; q <= q1; q += count) {
        const int b0 = q == q0 ? (lo & 31) : 0;
        const int b1 = q == q1 ? ((hi - 1) & 31) : 31;
        const uint32_t upto = b1 == 31 ? 0xFFFFFFFFu : ((1u << (b1 + 1)) - 1u);
        dlb[q] |= upto & ~((1u << b0) - 1u);
    }
}

__device__ __forceinline__ void dlb_clear(uint32_t *dlb, int c) { dlb[c >> 5] &= ~(1u << (c & 31)); }

// After the reversal of [pa..pb]: the two added edges border the path, and its
// two ends with their outer neighbours are the move's four cities, whose
// don't-look bits clear.  Whichever of the two paths was reversed, the edge
// before it is c1-c2 (successor side) or pred(c1)-pred(c2) (predecessor
// side), and the edge after it the other one.
__device__ __forceinline__ void finish_move(const TourView &tv, uint32_t *dlb, const Move &mv,
                                            int pa, int pb)
{
    const int ia = tv.prv(pa), ib = tv.nxt(pb);
    tv.edge[ia] = mv.side ? mv.d34 : mv.d12;
    tv.edge[pb] = mv.side ? mv.d12 : mv.d34;
    const int u = tv.tour[ia], v = tv.tour[pa], x = tv.tour[pb], y = tv.tour[ib];
    dlb_clear(dlb, u); dlb_clear(dlb, v); dlb_clear(dlb, x); dlb_clear(dlb, y);
}

// One warp applies move mv: the window's cities before mv.c1 get
// their bits set, then the shorter of the two paths between the removed edges
// is reversed and the move's edges and bits are updated.  Returns the first
// position of the reversed path and sets len to its length; the warp has
// synchronised, so every lane sees the finished move.
__device__ __forceinline__ int apply_move(const TourView &tv, uint32_t *dlb, const Move &mv, int l,
                                          int lane, int &len_out)
{
    const int n = tv.n;
    dlb_set_range(dlb, l, mv.c1, lane, 32);
    const int p = mv.p, q = mv.q;
    int pa, pb, ca, cb;  // path [pa..pb]; complement [ca..cb]
    if (mv.side == 0) {
        pa = tv.nxt(p); pb = q; ca = tv.nxt(q); cb = p;
    } else {
        pa = q; pb = tv.prv(p); ca = p; cb = tv.prv(q);
    }
    int len = pb - pa + 1;
    if (len <= 0) len += n;
    if (2 * len > n) {
        pa = ca;
        pb = cb;
        len = n - len;
    }
    reverse_path(tv, pa, pb, len, lane, 32);
    __syncwarp();
    if (lane == 0) finish_move(tv, dlb, mv, pa, pb);
    __syncwarp();
    len_out = len;
    return pa;
}

// Cities of a window whose search results (and footprints) are kept: the
// first city of each of the first MM_MAX warps.
constexpr int MM_MAX = 16;
// Moves one round may apply (their changed ranges are held in registers).
constexpr int MR_MAX = 8;

// Search results of the window's first cities, kept for the walk: res 0 = the
// city's bit was set (not searched), 1 = no move, 2 = a move (in the warp's
// move slot); fp = the footprint (find_move_warp).
struct RoundKeep {
    uint16_t fp[MM_MAX][33];
    int32_t res[MM_MAX];
    uint32_t hit[MM_MAX];  // bit i: the move of kept city i changes this city's footprint
    int32_t next, moves;
};

// The positions a move rewrites, widened by the footprint's one step: the
// reversed path [pa..pb] is the shorter one, as apply_move chooses it, and the
// range is pa - 2 .. pb + 2 (start ra, length rl, cyclic).
__device__ __forceinline__ void move_range(const Move &mv, int n, int &ra, int &rl)
{
    const int p = mv.p, q = mv.q;
    int pa, pb, ca;
    if (mv.side == 0) {
        pa = p + 1 == n ? 0 : p + 1; pb = q; ca = q + 1 == n ? 0 : q + 1;
    } else {
        pa = q; pb = p == 0 ? n - 1 : p - 1; ca = p;
    }
    int len = pb - pa + 1;
    if (len <= 0) len += n;
    if (2 * len > n) {
        pa = ca;
        len = n - len;
    }
    ra = pa >= 2 ? pa - 2 : pa - 2 + n;
    rl = len + 4 < n ? len + 4 : n;
}

// Warp j of the window (its kept city l + j): which moves of the earlier kept
// cities change its footprint (a skipped city's footprint is its own
// position: a move that clears its bit rewrites that position).
__device__ __forceinline__ uint32_t keep_hits(const RoundKeep &kp, const Move *s_move, int j, int k,
                                              int n, int lane)
{
    const int res = kp.res[j];
    const int p = kp.fp[j][0];  // every lane tests the city's own position (k may be 32)
    const int x = (res != 0 && lane < k) ? kp.fp[j][1 + lane] : p;
    uint32_t mask = 0;
    for (int i = 0; i < j; ++i) {
        if (kp.res[i] != 2) continue;
        int ra, rl;
        move_range(s_move[i], n, ra, rl);
        int dx = x - ra, dp = p - ra;
        if (dx < 0) dx += n;
        if (dp < 0) dp += n;
        if (__any_sync(0xFFFFFFFFu, dx < rl || dp < rl)) mask |= 1u << i;
    }
    return mask;
}

// Warp 0, after the round whose lowest improving city is `first` (window
// cities from l; city c's move, if any, is in slot (c - l) mod SL; cities below
// lim were kept in slot c - l): apply that
// move, then walk on through first + 1 .. lim - 1 while the kept results
// hold (no hit from a move applied so far).  Returns the next city to search
// and sets moves.
__device__ __forceinline__ int apply_moves(const TourView &tv, uint32_t *dlb, const Move *s_move,
                                           const RoundKeep &kp, int l, int first, int lim, int SL,
                                           int lane, int &moves)
{
    int len = 0;
    apply_move(tv, dlb, s_move[(first - l) & (SL - 1)], l, lane, len);
    if (first >= lim) {
        moves = 1;
        return first + 1;
    }
    uint32_t applied = 1u << (first - l);
    int nr = 1;
    int c = first + 1;
    for (; c < lim; ++c) {
        const int j = c - l;
        if (kp.hit[j] & applied) break;
        const int res = kp.res[j];
        if (res == 0) continue;  // its bit, set before, was not cleared
        if (res == 1) {          // no move on the new tour either
            if (lane == 0) dlb[c >> 5] |= 1u << (c & 31);
            __syncwarp();
            continue;
        }
        if (nr == MR_MAX) break;
        apply_move(tv, dlb, s_move[j], c, lane, len);
        applied |= 1u << j;
        ++nr;
    }
    moves = nr;
    return c;
}

// PAIR: k <= 16 and at most 16 warps; each warp searches two cities at a time
// (a half each), so a window's first 16 cities take 8 warps.
template <bool XY, bool STAGED, bool IB, bool PAIR>
__global__ void __launch_bounds__(1024, 1) k_two_opt(const TwoOptArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n, tid = threadIdx.x, W = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, NW = W >> 5;
    // cities searched at a time: one a warp, two with PAIR; city c of a window
    // from l is searched in slot (c - l) mod SL (its move slot), by warp
    // slot / S and, with PAIR, its half slot % 2
    constexpr int S = PAIR ? 2 : 1;
    const int SL = S * NW;
    const int slot0 = S * warp + (PAIR ? (lane >> 4) : 0);
    const int gl = PAIR ? (lane & 15) : lane;  // lane within the searching group
    // cities in the first window after a move: one a slot, as far as results are kept
    const int first_window = SL < MM_MAX ? SL : MM_MAX;
    const Layout L = Layout::make(n, a.k, STAGED);
    TourView tv;
    tv.n = n;
    tv.edge = reinterpret_cast<int32_t *>(smem + L.edge);
    tv.tour = reinterpret_cast<int32_t *>(smem + L.tour);
    tv.pos = reinterpret_cast<int32_t *>(smem + L.pos);
    uint32_t *s_dlb = reinterpret_cast<uint32_t *>(smem + L.dlb);
    const int dlb_words = (n + 31) >> 5;
    const Geometry<XY, STAGED> g{a, reinterpret_cast<const int2 *>(smem + L.xy),
                                 reinterpret_cast<const uint16_t *>(smem + L.nn)};
    __shared__ int s_first[3];
    __shared__ Move s_move[32];  // per warp
    __shared__ RoundKeep s_keep;
    const int mm = SL < MM_MAX ? SL : MM_MAX;  // window cities whose results are kept
    __shared__ int s_red[32];
    __shared__ unsigned long long s_best;

    if constexpr (STAGED) {
        int2 *sxy = reinterpret_cast<int2 *>(smem + L.xy);
        for (int i = tid; i < n; i += W) sxy[i] = __ldg(a.xy + i);
        const uint4 *src = reinterpret_cast<const uint4 *>(a.nn16);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + L.nn);
        const int chunks = (2 * n * a.k + 15) / 16;  // the list buffer is padded to 16 bytes
        for (int i = tid; i < chunks; i += W) dst[i] = __ldg(src + i);
    }

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
            tv.edge[i] = g.d(c, row[i + 1 == n ? 0 : i + 1]);
        }
        if (tid < 3) s_first[tid] = INT_MAX;
        __syncthreads();
        // every move shortens the tour by >= 1, so the search ends; the cap
        // (far above the moves a tour needs) only guards against a defect
        const long long cap = g_two_opt_cap > 0 ? g_two_opt_cap : 64LL * n;
        long long total = 0;
        bool capped = false;
        uint32_t round = 0;  // selects the key slot
        for (;;) {  // runs
            for (int i = tid; i < dlb_words; i += W) s_dlb[i] = 0;
            __syncthreads();
            long long run_moves = 0;
            bool improved = true;
            while (improved && !capped) {  // passes
                improved = false;
                int l = 0;
                int w = first_window;  // cities in the window; doubles while none has a move
                while (l < n) {  // windows
                    const int wend = l + w < n ? l + w : n;
                    int mine = INT_MAX;
                    // this group's cities l + slot0, l + slot0 + SL, ... up to its
                    // first move; the loop runs while either half of the warp has one
                    int c1 = l + slot0;
                    bool live = c1 < wend;
                    bool first_city = true;
                    while (__any_sync(0xFFFFFFFFu, live)) {  // warp-uniform
                        const bool keep = live && first_city && slot0 < mm;
                        const bool skip = live && dlb_get(s_dlb, c1);
                        if (keep && skip && gl == 0) {
                            s_keep.res[slot0] = 0;
                            s_keep.fp[slot0][0] = (uint16_t)tv.pos[c1];
                        }
                        const bool act = live && !skip;
                        Move mv;
                        const bool found = find_move_warp<XY, STAGED, PAIR>(
                            a, g, tv, act ? c1 : 0, lane, act, mv, (keep && act) ? s_keep.fp[slot0] : nullptr);
                        if (keep && act && gl == 0) s_keep.res[slot0] = found ? 2 : 1;
                        if (found) {  // (act, since nothing is found otherwise)
                            if (gl == 0) s_move[slot0] = mv;
                            mine = c1;
                            live = false;
                        }
                        c1 += SL;
                        live = live && c1 < wend;
                        first_city = false;
                    }
                    int *slot = s_first + round % 3;
                    if (gl == 0 && mine != INT_MAX) atomicMin(slot, mine);
                    __syncthreads();
                    const int first = *slot;
                    if (tid == 0) s_first[(round + 2) % 3] = INT_MAX;  // no one reads it for two rounds
                    ++round;
                    if (first == INT_MAX) {
                        dlb_set_range(s_dlb, l, wend, tid, W);
                        l = wend;
                        w = w * 2 < W ? w * 2 : W;
                        continue;
                    }
                    // cities [l, first) were evaluated without a move (every group
                    // stopped at its own first move, so all of them were reached);
                    // city c was searched in slot (c - l) mod SL
                    const int lim = wend < l + mm ? wend : l + mm;
                    if (first < lim) {  // the kept cities after first: hits, a warp each
                        for (int j = warp; j < mm; j += NW) {
                            if (l + j > first && l + j < lim) {
                                const uint32_t h = keep_hits(s_keep, s_move, j, a.k, n, lane);
                                if (lane == 0) s_keep.hit[j] = h;
                            }
                        }
                        __syncthreads();
                    }
                    if (warp == 0) {
                        int moves = 0;
                        const int next = apply_moves(tv, s_dlb, s_move, s_keep, l, first, lim, SL,
                                                     lane, moves);
                        if (lane == 0) {
                            s_keep.next = next;
                            s_keep.moves = moves;
                        }
                    }
                    improved = true;
                    __syncthreads();
                    const int moves = s_keep.moves;
                    run_moves += moves;
                    l = s_keep.next;
                    w = first_window;
                    total += moves;
                    if (total > cap) {
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
    const Geometry<XY, false> g{a, nullptr, nullptr};
    const size_t total = (size_t)a.n * a.k;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / a.k);
        nnd[e] = g.d(c, a.nn[e]);
    }
}

template <bool XY, bool STAGED, bool IB, bool PAIR>
cudaError_t launch_pair(const TwoOptArgs &a, int grid, int threads, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_two_opt<XY, STAGED, IB, PAIR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_two_opt<XY, STAGED, IB, PAIR><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

// Two cities a warp when the lists are at most 16 long and the slots (two a
// warp) fit the 32 move slots.
template <bool XY, bool STAGED, bool IB>
cudaError_t launch_one(const TwoOptArgs &a, int grid, int threads, size_t smem, cudaStream_t s)
{
    if (a.k <= 16 && threads <= 512) return launch_pair<XY, STAGED, IB, true>(a, grid, threads, smem, s);
    return launch_pair<XY, STAGED, IB, false>(a, grid, threads, smem, s);
}

}  // namespace

size_t two_opt_smem(int n, int k, bool staged) { return Layout::make(n, k, staged).total; }

bool two_opt_fits(int n, int k, bool staged, size_t smem_optin)
{
    // + the kernel's static shared memory (move slots, the kept search
    // results, reduction words: 2,048 bytes) with room to spare
    return two_opt_smem(n, k, staged) + 2304 <= smem_optin;
}

cudaError_t launch_neighbour_dist(const TwoOptArgs &a, int32_t *nnd, cudaStream_t s)
{
    if (a.xy)
        k_neighbour_dist<true><<<256, 256, 0, s>>>(a, nnd);
    else
        k_neighbour_dist<false><<<256, 256, 0, s>>>(a, nnd);
    return cudaGetLastError();
}

cudaError_t set_two_opt_move_cap(long long cap)
{
    const long long v = cap > 0 ? cap : 0;
    return cudaMemcpyToSymbol(g_two_opt_cap, &v, sizeof(v));
}

cudaError_t launch_two_opt(const TwoOptArgs &a, bool iteration_best, int num_sms, int smem_optin,
                           cudaStream_t s)
{
    if (iteration_best) {
        // one tour, one CTA: stage coordinates and lists when they fit.  16
        // warps: windows of up to 512 cities; on the clustered n = 3800 tours
        // 512 threads took 3.65 ms a launch, 1024 took 3.76 and 256 took 3.95
        const bool staged = a.xy && two_opt_fits(a.n, a.k, true, (size_t)smem_optin);
        const size_t smem = two_opt_smem(a.n, a.k, staged);
        constexpr int IB_THREADS = 512;
        if (staged) return launch_one<true, true, true>(a, 1, IB_THREADS, smem, s);
        if (a.xy) return launch_one<true, false, true>(a, 1, IB_THREADS, smem, s);
        return launch_one<false, false, true>(a, 1, IB_THREADS, smem, s);
    }
    // every tour: one CTA of 256 threads per tour, many per SM
    const size_t smem = two_opt_smem(a.n, a.k, false);
    const int grid = a.m < num_sms * 8 ? a.m : num_sms * 8;
    if (a.xy) return launch_one<true, false, false>(a, grid, 256, smem, s);
    return launch_one<false, false, false>(a, grid, 256, smem, s);
}

}  // namespace mmas
