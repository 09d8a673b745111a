// Solution construction (Alg. 1, inner loops) with tour lengths fused in.
//
// One warp builds one ant's tour.  At each of the n-1 steps the warp scores the
// unvisited nodes of Eq. (1)'s neighbourhood with weighted-reservoir keys
// log2(r) / w (Alg. 4, Sec. 4.2.2), reduces them with one redux.max and one
// redux.min (ties -> lower node id), marks the winner in a bitmask tabu
// (Sec. 4.1) and appends it to the tour.
//
//  - Candidate-list mode (cl in 1..32, Sec. 4.3): lane c scores candidate
//    slot c.  The slot's uniform depends on (iteration, ant, step, slot) only,
//    so one Philox call yields the draws of four consecutive steps and the
//    log2 of each is taken off the step-to-step dependency chain.  When every
//    candidate is visited, the fallback scans the unvisited nodes of the row.
//  - Whole-row mode (cl = 0): lane l scores nodes 4c..4c+3 for c = l, l+32, ...,
//    reading 16 bytes of 1/choice_info per chunk and one Philox call per chunk.
//
// The table a step reads (n x cl ids + reciprocal weights, or the n x ld
// reciprocal weight matrix) is copied into shared memory once per CTA with the
// bulk-copy engine when it fits; each CTA then runs ceil(m / #SMs) ants.
// The tabu of an ant lives in registers (lane l holds nodes 32l..32l+31) when
// n <= 1024, otherwise in the warp's slice of shared memory.
// Tour entries are buffered one per lane and written as 128-byte rows every 32
// steps; each lane then adds the length of its edge.
#include "internal.cuh"

namespace mmas {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr unsigned long long STAGE_LIMIT_NS = 2000000000ull;  // 2 s
constexpr uint32_t BULK_CHUNK = 32768u;

enum { CAND = 0, ROW = 1 };

template <bool XY>
__device__ __forceinline__ int32_t edge_len(const ConstructArgs &a, int u, int v)
{
    if constexpr (XY)
        return euc2d_exact(__ldg(a.xy + u), __ldg(a.xy + v));
    else
        return __ldg(a.dist + (size_t)u * a.ld + v);
}

// Bitmask tabu (Sec. 4.1, "BT"): mark / is_visited in O(1).
template <bool REGMASK>
struct Tabu {
    uint32_t reg = 0;          // REGMASK: word `lane` of the bitmask
    uint32_t *w = nullptr;     // otherwise: this warp's words in shared memory
    int nw = 0;

    __device__ __forceinline__ void clear(int lane)
    {
        if constexpr (REGMASK) {
            reg = 0;
        } else {
            for (int q = lane; q < nw; q += 32) w[q] = 0;
            __syncwarp();
        }
    }
    __device__ __forceinline__ void mark(int lane, int v)
    {
        if constexpr (REGMASK) {
            if (lane == (v >> 5)) reg |= 1u << (v & 31);
        } else {
            if (lane == 0) w[v >> 5] |= 1u << (v & 31);
            __syncwarp();
        }
    }
    // The bitmask word that holds node v.  Every lane of the warp must call it.
    __device__ __forceinline__ uint32_t word_of(int v) const
    {
        if constexpr (REGMASK)
            return __shfl_sync(FULL, reg, (v >> 5) & 31);
        else
            return w[v >> 5];
    }
    // Word q for q in [0, nw), read by the lane that scans it.
    __device__ __forceinline__ uint32_t word_at(int q) const
    {
        if constexpr (REGMASK)
            return reg;  // q == lane when n <= 1024
        else
            return w[q];
    }
};

__device__ __forceinline__ uint32_t pick_word(const uint4 &r, int e)
{
    return e == 0 ? r.x : (e == 1 ? r.y : (e == 2 ? r.z : r.w));
}

// Fallback when every candidate of `cur` is visited (fallback = 0): the
// unvisited node with the largest choice_info, ties -> lower id.  With
// fallback = 1: reservoir keys over all unvisited nodes (whole-row stream).
template <bool REGMASK>
__device__ __forceinline__ int fallback_pick(const ConstructArgs &a, const Tabu<REGMASK> tb,
                                          int lane, int cur, int t, int ant, uint32_t it)
{
    const float *row = a.wmat + (size_t)cur * a.ld;
    uint32_t bk = 0, bj = 0xFFFFFFFFu;
    for (int q0 = 0; q0 < tb.nw; q0 += 32) {
        const int q = q0 + lane;
        uint32_t un = 0;
        if (q < tb.nw) {
            un = ~tb.word_at(q);
            if (q == tb.nw - 1 && (a.n & 31)) un &= (1u << (a.n & 31)) - 1u;
        }
        while (un) {
            const int b = __ffs(un) - 1;
            un &= un - 1;
            const int j = (q << 5) + b;
            const float w = __ldg(row + j);
            uint32_t kk;
            if (a.fallback == 0) {
                kk = ord_key(w);
            } else {
                const uint4 r = philox10(make_uint4(0x80000000u | ((uint32_t)j >> 2), (uint32_t)t,
                                                    (uint32_t)ant, it),
                                         a.key0, a.key1);
                const float lg = log2f(unit_open(pick_word(r, j & 3)));
                kk = ord_key(__fmul_rn(lg, __frcp_rn(w)));
            }
            if (kk > bk) {
                bk = kk;
                bj = (uint32_t)j;
            }
        }
    }
    const uint32_t mx = __reduce_max_sync(FULL, bk);
    if (mx == 0u) {
        if (lane == 0) atomicOr(&a.sc->err, ERR_NO_UNVISITED);
        return cur;
    }
    return (int)__reduce_min_sync(FULL, bk == mx ? bj : 0xFFFFFFFFu);
}

// One candidate-list step: lane c scores slot c of cur's list.
template <bool REGMASK>
__device__ __forceinline__ int select_cand(const ConstructArgs &a, const uint16_t *cc,
                                           const float *cw, const Tabu<REGMASK> &tb, int lane,
                                           int cur, float lg, int t, int ant, uint32_t it,
                                           uint32_t &fbn)
{
    const bool act = lane < a.cl;
    uint32_t v = 0;
    float wi = 0.0f;
    if (act) {
        const int idx = cur * a.cl + lane;
        v = cc[idx];
        wi = cw[idx];
    }
    const uint32_t word = tb.word_of((int)v);
    const bool ok = act && !((word >> (v & 31)) & 1u);
    const uint32_t k = ok ? ord_key(__fmul_rn(lg, wi)) : 0u;
    const uint32_t mx = __reduce_max_sync(FULL, k);
    if (mx != 0u) return (int)__reduce_min_sync(FULL, k == mx ? v : 0xFFFFFFFFu);
    ++fbn;
    return fallback_pick<REGMASK>(a, tb, lane, cur, t, ant, it);
}

// One whole-row step: lane l scores nodes 4c..4c+3 for c = l, l + 32, ...
template <bool REGMASK>
__device__ __forceinline__ int select_row(const ConstructArgs &a, const float *W,
                                          const Tabu<REGMASK> &tb, int lane, int cur, int t,
                                          int ant, uint32_t it)
{
    const float *row = W + (size_t)cur * a.ld;
    const int nch = (a.n + 3) >> 2;
    uint32_t bk = 0, bv = 0xFFFFFFFFu;
    for (int c0 = 0; c0 < nch; c0 += 32) {
        const int c = c0 + lane;
        const int v0 = c << 2;
        const uint32_t word = tb.word_of(v0 < a.n ? v0 : a.n - 1);
        if (c < nch) {
            const uint32_t bits = (word >> (v0 & 31)) & 0xFu;
            if (bits != 0xFu) {
                const uint4 r = philox10(
                    make_uint4(0x80000000u | (uint32_t)c, (uint32_t)t, (uint32_t)ant, it), a.key0,
                    a.key1);
                const float4 wi = *reinterpret_cast<const float4 *>(row + v0);
                const float wv[4] = {wi.x, wi.y, wi.z, wi.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int v = v0 + e;
                    if (v < a.n && !((bits >> e) & 1u)) {
                        const float lg = log2f(unit_open(pick_word(r, e)));
                        const uint32_t kk = ord_key(__fmul_rn(lg, wv[e]));
                        if (kk > bk) {
                            bk = kk;
                            bv = (uint32_t)v;
                        }
                    }
                }
            }
        }
    }
    const uint32_t mx = __reduce_max_sync(FULL, bk);
    if (mx == 0u) {
        if (lane == 0) atomicOr(&a.sc->err, ERR_NO_UNVISITED);
        return cur;
    }
    return (int)__reduce_min_sync(FULL, bk == mx ? bv : 0xFFFFFFFFu);
}

template <int MODE, bool STAGED, bool REGMASK, bool XY>
__global__ void __launch_bounds__(1024, 1) k_construct(const ConstructArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;

    const float *cw = (MODE == CAND) ? a.cwinv : a.wmat;
    const uint16_t *cc = a.cand16;
    size_t off = 0;
    if constexpr (STAGED) {
        unsigned char *s_w = smem;
        off = a.stage_w_bytes;
        unsigned char *s_c = smem + off;
        off += a.stage_c_bytes;
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem + off);
        off += 16;
        if (threadIdx.x == 0) mbar_init(bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(bar, a.stage_w_bytes + a.stage_c_bytes);
            const unsigned char *src_w = reinterpret_cast<const unsigned char *>(cw);
            for (uint32_t o = 0; o < a.stage_w_bytes; o += BULK_CHUNK)
                bulk_copy_g2s(s_w + o, src_w + o, min(BULK_CHUNK, a.stage_w_bytes - o), bar);
            const unsigned char *src_c = reinterpret_cast<const unsigned char *>(a.cand16);
            for (uint32_t o = 0; o < a.stage_c_bytes; o += BULK_CHUNK)
                bulk_copy_g2s(s_c + o, src_c + o, min(BULK_CHUNK, a.stage_c_bytes - o), bar);
        }
        if (!mbar_wait_bounded(bar, 0, STAGE_LIMIT_NS)) {
            if (threadIdx.x == 0) atomicOr(&a.sc->err, ERR_STAGE_TIMEOUT);
            // let copies still in flight land before the CTA's memory is released
            mbar_wait_bounded(bar, 0, STAGE_LIMIT_NS);
            return;
        }
        cw = reinterpret_cast<const float *>(s_w);
        cc = reinterpret_cast<const uint16_t *>(s_c);
    }

    Tabu<REGMASK> tb;
    tb.nw = (a.n + 31) >> 5;
    if constexpr (!REGMASK) tb.w = reinterpret_cast<uint32_t *>(smem + off) + (size_t)warp * tb.nw;

    const uint32_t it = (uint32_t)a.iter[0];
    const int stride = gridDim.x * warps;
    for (int ant = blockIdx.x * warps + warp; ant < a.m; ant += stride) {
        // Alg. 1: the first node is drawn uniformly
        const uint4 s4 = philox10(make_uint4(0xFFFFFFFFu, 0u, (uint32_t)ant, it), a.key0, a.key1);
        const int start = (int)(((unsigned long long)s4.x * (unsigned)a.n) >> 32);
        tb.clear(lane);
        tb.mark(lane, start);
        int cur = start;
        int twin = start;      // this lane's entry of the current 32-step window
        int prev_last = -1;    // last node of the previous window
        int acc = 0;           // this lane's share of the tour length
        uint32_t fbn = 0;
        int32_t *trow = a.tours + (size_t)ant * a.ld;

        for (int g = 0; (g << 2) < a.n; ++g) {
            float lg0 = 0.f, lg1 = 0.f, lg2 = 0.f, lg3 = 0.f;
            if constexpr (MODE == CAND) {
                if (lane < a.cl) {
                    const uint4 r = philox10(
                        make_uint4((uint32_t)lane, (uint32_t)g, (uint32_t)ant, it), a.key0, a.key1);
                    lg0 = log2f(unit_open(r.x));
                    lg1 = log2f(unit_open(r.y));
                    lg2 = log2f(unit_open(r.z));
                    lg3 = log2f(unit_open(r.w));
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int t = (g << 2) + j;
                if (t == 0) continue;
                if (t >= a.n) break;
                int next;
                if constexpr (MODE == CAND) {
                    const float lg = j == 0 ? lg0 : (j == 1 ? lg1 : (j == 2 ? lg2 : lg3));
                    next = select_cand<REGMASK>(a, cc, cw, tb, lane, cur, lg, t, ant, it, fbn);
                } else {
                    next = select_row<REGMASK>(a, cw, tb, lane, cur, t, ant, it);
                }
                tb.mark(lane, next);
                if (lane == (t & 31)) twin = next;
                if ((t & 31) == 31 || t == a.n - 1) {
                    const int t0 = t & ~31, cnt = (t & 31) + 1;
                    if (lane < cnt) trow[t0 + lane] = twin;
                    int prev = __shfl_up_sync(FULL, twin, 1);
                    if (lane == 0) prev = prev_last;
                    if (lane < cnt && prev >= 0) acc += edge_len<XY>(a, prev, twin);
                    prev_last = __shfl_sync(FULL, twin, 31);
                }
                cur = next;
            }
        }
        if (lane == 0) acc += edge_len<XY>(a, cur, start);  // close the cycle
        const int total = (int)__reduce_add_sync(FULL, (unsigned)acc);
        if (lane == 0) {
            a.lens[ant] = total;
            if (fbn) atomicAdd(&a.sc->fallback_steps, (unsigned long long)fbn);
        }
    }
}

using KernelFn = void (*)(const ConstructArgs);

KernelFn pick_kernel(int mode, int staged, int regmask, int xy)
{
    static const KernelFn table[16] = {
        k_construct<CAND, false, false, false>, k_construct<CAND, false, false, true>,
        k_construct<CAND, false, true, false>,  k_construct<CAND, false, true, true>,
        k_construct<CAND, true, false, false>,  k_construct<CAND, true, false, true>,
        k_construct<CAND, true, true, false>,   k_construct<CAND, true, true, true>,
        k_construct<ROW, false, false, false>,  k_construct<ROW, false, false, true>,
        k_construct<ROW, false, true, false>,   k_construct<ROW, false, true, true>,
        k_construct<ROW, true, false, false>,   k_construct<ROW, true, false, true>,
        k_construct<ROW, true, true, false>,    k_construct<ROW, true, true, true>,
    };
    return table[(mode << 3) | (staged << 2) | (regmask << 1) | xy];
}

}  // namespace

cudaError_t plan_construct(const ConstructArgs &a, int num_sms, size_t smem_optin,
                           ConstructPlan *plan)
{
    const bool row = a.cl == 0;
    const int nw = (a.n + 31) / 32;
    plan->regmask = a.n <= 1024;
    const size_t table = row ? (size_t)a.n * a.ld * sizeof(float)
                             : (size_t)a.stage_w_bytes + a.stage_c_bytes;
    int w = (a.m + num_sms - 1) / num_sms;
    w = w < 1 ? 1 : (w > 32 ? 32 : w);
    const size_t masks = plan->regmask ? 0 : (size_t)w * nw * sizeof(uint32_t);
    const size_t need = table + 16 + masks;
    if (need <= smem_optin && table < (1u << 30)) {
        plan->staged = 1;
        plan->warps = w;
        plan->grid = (a.m + w - 1) / w;
        plan->smem = need;
    } else {
        plan->staged = 0;
        plan->warps = 4;
        plan->grid = (a.m + 3) / 4;
        plan->smem = plan->regmask ? 0 : (size_t)4 * nw * sizeof(uint32_t);
    }
    KernelFn k = pick_kernel(row ? ROW : CAND, plan->staged, plan->regmask, a.xy != nullptr);
    return cudaFuncSetAttribute(reinterpret_cast<const void *>(k),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan->smem);
}

cudaError_t launch_construct(const ConstructArgs &a, const ConstructPlan &plan, cudaStream_t s)
{
    ConstructArgs b = a;
    if (!plan.staged) {
        b.stage_w_bytes = 0;
        b.stage_c_bytes = 0;
    } else if (a.cl == 0) {
        b.stage_w_bytes = (uint32_t)((size_t)a.n * a.ld * sizeof(float));
        b.stage_c_bytes = 0;
    }
    KernelFn k = pick_kernel(a.cl == 0 ? ROW : CAND, plan.staged, plan.regmask, a.xy != nullptr);
    k<<<plan.grid, plan.warps * 32, plan.smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace mmas
