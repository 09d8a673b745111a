// Internal declarations shared by the translation units of libmmas.so.
// Device helpers, the device-resident scalar block, launch-argument structs and
// the host-side launchers.  Nothing here is part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace mmas {

// ---------------------------------------------------------------------------
// Error bits raised on the device; the host reads them at synchronising calls.
// ---------------------------------------------------------------------------
enum : uint32_t {
    ERR_STAGE_TIMEOUT = 1u,   // a shared-memory staging wait gave up
    ERR_NO_UNVISITED = 2u,    // a selection found no unvisited node (inconsistent tabu)
    ERR_LS_CAP = 4u,          // a local search exceeded its move cap and stopped
    ERR_BAD_TOUR = 8u,        // a device-side tour handed to the update was not a permutation
};

// Device-resident scalars of one colony.  Kernels read and write them, so a
// captured CUDA graph replays whole iterations without host round trips.
struct Scalars {
    int32_t iter;          // index of the next iteration (keys the random draws)
    int32_t gb_len;        // global best length, INT32_MAX before the first iteration
    int32_t ib_len;        // last iteration best length (-1 before the first)
    int32_t ib_ant;        // last iteration best ant
    float tmin, tmax;      // trail limits
    float delta;           // deposit amount of the pending update (float 1/C)
    int32_t dep_len;       // length of the tour being deposited
    uint32_t err;          // ERR_* bits
    uint32_t done;         // CTAs of the scoring kernel that finished (last-block election)
    unsigned long long fallback_steps;  // cumulative candidate-list fallbacks
    unsigned long long fallback_scans;  // of those, the ones that scanned the whole row
    long long nn_len;      // nearest-neighbour tour length
    long long iterations;  // completed iterations
};

// ---------------------------------------------------------------------------
// Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// Ten rounds; each multiplies words 0 and 2 by the round multipliers, mixes
// the high halves with words 1 and 3 and the key, and bumps the key by the
// Weyl increments.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Rounds [R0, R1) of the same generator on counter c, for spreading one call
// over several steps of a dependent chain (round r uses key + r * Weyl).
template <int R0, int R1>
__device__ __forceinline__ void philox_rounds(uint4 &c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = R0; r < R1; ++r) {
        const uint32_t rk0 = k0 + (uint32_t)r * 0x9E3779B9u;
        const uint32_t rk1 = k1 + (uint32_t)r * 0xBB67AE85u;
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;  // one wide multiply
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk0, (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk1, (uint32_t)p0);
    }
}

// The same rounds with the per-round keys precomputed (rk0[r] = k0 + r W0,
// rk1[r] = k1 + r W1), e.g. held in kernel parameters.
template <int R0, int R1>
__device__ __forceinline__ void philox_rounds_rk(uint4 &c, const uint32_t *rk0, const uint32_t *rk1)
{
#pragma unroll
    for (int r = R0; r < R1; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk0[r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk1[r], (uint32_t)p0);
    }
}

// r = ((x >> 9) + 1/2) * 2^-23, exactly representable, in (0, 1): the float
// with exponent 0 and mantissa x >> 9 is 1 + k 2^-23 (k = x >> 9), and
// subtracting 1 - 2^-24 from it is exact (Sterbenz), leaving k 2^-23 + 2^-24.
__device__ __forceinline__ float unit_open(uint32_t x)
{
    return __fsub_rn(__uint_as_float(0x3F800000u | (x >> 9)), 0.99999994039535522461f);
}

// log2 of a candidate draw r = ((x >> 9) + 1/2) 2^-23 in (0, 1), to within
// DRAW_LOG2_MAX_REL relative on that grid of 2^23 values (every one of them is
// checked by mmas_debug_draw_log2_error).  Below r = 0.55 the hardware's
// approximate log2, whose error there is at most 2^-22.6 absolute on [0.5, 2)
// and 2 ulp below 0.5, so about 2.4e-7 relative at most (|log2 r| > 0.86).
// From 0.55 up, where log2 r nears 0 and an absolute bound is useless:
// log2(1 + f) with f = r - 1 (exact by Sterbenz) from the series
// ln((1 + s) / (1 - s)) = 2 (s + s^3/3 + s^5/5 + ...), s = f / (2 + f)
// (Abramowitz and Stegun 4.1.28), |s| < 0.291: six terms leave a truncation
// below 3e-8 relative, the fast division 2 ulp.  Measured over every value:
// 2.55e-7 at most (the library's log2f: 1.07e-7).  The reservoir keys only
// need their order, so this relative accuracy is what the selection depends on.
constexpr double DRAW_LOG2_MAX_REL = 2.6e-7;
__device__ __forceinline__ float draw_log2(float r)
{
    const float f = __fsub_rn(r, 1.0f);
    const float s = __fdividef(f, __fadd_rn(2.0f, f));
    const float s2 = __fmul_rn(s, s);
    // (2 / ln 2) / (2i + 1), i = 5 .. 0
    float p = __fmaf_rn(s2, 0.26230819f, 0.32059890f);
    p = __fmaf_rn(p, s2, 0.41219858f);
    p = __fmaf_rn(p, s2, 0.57707802f);
    p = __fmaf_rn(p, s2, 0.96179669f);
    p = __fmaf_rn(p, s2, 2.88539008f);
    const float near1 = __fmul_rn(s, p);
    const float far = __log2f(r);
    return r < 0.55f ? far : near1;
}

// Order-preserving map of a negative float to uint32 (larger float -> larger
// code), for the reservoir keys log2(r) / w, which are negative (r < 1, w > 0);
// the codes are >= 1, so 0 still marks "no candidate".
__device__ __forceinline__ uint32_t neg_key(float f) { return ~__float_as_uint(f); }

// Order-preserving map of a float to uint32 (larger float -> larger code).
// Codes are >= 1 for every non-NaN float, so 0 marks "no candidate".
__device__ __forceinline__ uint32_t ord_key(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Trail limits (after Stuetzle and Hoos, as Sec. 5 states): tau_max = 1/(rho C),
// tau_min = tau_max (1 - p)/((n/2 - 1) p), capped at tau_max; double, stored float.
__device__ __forceinline__ void trail_limits(int32_t n, double rho, double p_root, long long cost, float *tmax,
                             float *tmin)
{
    const double tx = __ddiv_rn(1.0, __dmul_rn(rho, (double)cost));
    const double avg = __ddiv_rn((double)n, 2.0);
    double tn = __ddiv_rn(__dmul_rn(tx, __dsub_rn(1.0, p_root)),
                          __dmul_rn(__dsub_rn(avg, 1.0), p_root));
    if (tn > tx) tn = tx;
    *tmax = (float)tx;
    *tmin = (float)tn;
}

// ---------------------------------------------------------------------------
// mbarrier + bulk asynchronous copy (TMA engine, non-tensor form) helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Copy `bytes` (multiple of 16, both addresses 16-byte aligned) from global to
// this CTA's shared memory; completion is signalled on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` for at most `limit_ns`; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns)
{
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Launch arguments
// ---------------------------------------------------------------------------
struct ConstructArgs {
    int32_t n, m, cl, ld, fallback;
    int32_t ant_offset;        // global index of ant 0 (keys the draws)
    uint32_t key0, key1;
    uint32_t rk0[10], rk1[10];  // Philox round keys: key + r * Weyl increment
    const int32_t *iter;       // device iteration index
    const uint16_t *cand16;    // [n][cl] candidate ids
    const float *cwinv;        // [n][cl] 1 / choice_info of each candidate
    const float *wmat;         // [n][ld] choice_info (cl > 0) or 1/choice_info (cl == 0)
    int32_t *tours;            // [m][ld]
    Scalars *sc;
    uint32_t stage_w_bytes;    // bytes of the staged weight table (16-byte multiple)
    uint32_t stage_c_bytes;    // bytes of the staged id table (16-byte multiple)
    int32_t stage_rows;        // rows of the candidate table staged (n when whole)
    int32_t sel;               // whole-row selection: 0 reservoir sampling, 1 roulette wheel
    int32_t ct;                // whole-row tabu: 0 bitmask, 1 compact list
    // greedy-fallback reach list (candidate-list mode, fallback 0; xe = 0: none,
    // else xe <= REACH_MAX):
    // per row the xe nearest nodes with this iteration's choice_info, and a
    // bound on the choice_info of every node outside the list
    int32_t xe;
    const uint2 *xlw;          // [n][xe] {float bits of choice_info, node}
    const float *xlb;          // [n]
    const uint2 *xxw;          // [n][REACH_EXTRA] nodes outside the list above the trail floor
    const int32_t *xxn;        // [n] how many of them are stored
    // far list (rows of n >= REACH_FAR_MIN_N), in device memory, or nullptr:
    // none.  Behind one pointer so the steps' fallback calls stay as light as
    // without it
    const struct FarList *far;
};

// Far list of a colony's greedy fallback: per row the nodes ranked REACH_MAX +
// 1 .. REACH_FAR by (distance, id), at entries REACH_MAX .. of a row of xf16
// (pitch fp = REACH_FAR; the first REACH_MAX entries repeat the reach list),
// and a bound on the choice_info of every node beyond them.
struct FarList {
    const uint16_t *xf16;  // [n][fp]
    const float *xfb;      // [n]
    int32_t fp;
    int32_t pad;
};

// Longest reach list of the greedy fallback (lane l of a warp holds entries
// l, l + 32, l + 64, l + 96).
constexpr int REACH_MAX = 128;
// Nodes outside the reach list whose trail is above tau_min, stored per row
// beside it (lane l holds one); the bound covers the rest.
constexpr int REACH_EXTRA = 32;
// Far list of the greedy fallback: a row's nearest REACH_FAR nodes, for rows of
// at least REACH_FAR_MIN_N nodes.  When every node of the reach list is
// visited, the next unvisited ones usually rank below REACH_FAR: their
// choice_info is gathered from the row and compared with a bound on the rest,
// which replaces most row scans (uniform n = 18,500: 88% of the fallbacks are
// decided by the 128 nearest, 98.7% by the 1024 nearest).  Shorter rows scan
// in few round trips, and there the list cost more than it saved (n = 5,000:
// 6.29 ms of construction with it, 6.14 without).
constexpr int REACH_FAR = 1024;
// The fused pass gives each row a CTA up to this many rows, else a warp.
constexpr int UPDATE_CTA_MAX_N = 8192;
// Far lists only for colonies whose rows the warp form updates (it computes
// their bound; the CTA form, used for fewer rows, has no far-list code).
constexpr int REACH_FAR_MIN_N = UPDATE_CTA_MAX_N + 1;
static_assert((REACH_FAR - REACH_MAX) % 64 == 0 && REACH_FAR_MIN_N > REACH_FAR,
              "far-list entries come two to a word, 32 words a warp round; rows hold REACH_FAR nodes");

// One unit of batched construction: ants first .. first+count-1 of a colony.
struct BatchChunk {
    int32_t colony, first, count;
};

struct ConstructPlan {
    int staged;     // 0: no staging; 1: the whole table in shared memory; 2: its first stage_rows rows
    int stage_rows;
    int tw;         // tabu words per lane in registers (1, 2, 4; n <= 1024 tw), 0: shared memory
    int wide;       // 1: 32 warps per CTA (MAXT 1024): most rows read from L2
    int longl;      // 1: 32 < cl <= 64, two candidate slots per lane (k_construct_long)
    int cons_warps; // warps building tours (one ant each) per CTA
    int gen_warps;  // reserved (0)
    int grid;
    size_t smem;    // dynamic shared memory bytes
};

struct BestArgs {
    int32_t n, m, ld, deposit, advance;
    double rho;        // evaporation rate as double
    double p_root;     // p_best^(1/n)
    const int32_t *lens;
    const int32_t *tours;  // [m][ld]
    int32_t *gb_tour;      // [n]
    int2 *nbr;             // [n]: successor and predecessor in the deposited tour
    Scalars *sc;
    const uint32_t *skip;  // nullptr, or a device flag: when set the step does nothing
};

struct ScoreArgs {
    int32_t n, m, ld, best;
    const int32_t *tours;  // [m][ld]
    const int2 *xy;        // coordinates, or nullptr (then dist)
    const int32_t *dist;   // [n][ld]
    int32_t *lens;         // [m]
    BestArgs b;            // used by the last CTA when best != 0
};

struct UpdateArgs {
    int32_t n, ld, cl, fullrow, evaporate;
    int32_t recip;     // whole-row mode: store 1/choice_info (reservoir sampling) or choice_info
    float persist;     // float(1 - rho)
    float alpha;
    const float *eb;   // [n][ld]
    float *tau;        // [n][ld]
    float *wmat;       // [n][ld]
    const int32_t *cand32;  // [n][cl]
    float *cwinv;      // [n][cl]
    const int2 *nbr;   // [n] or nullptr (no deposit)
    Scalars *sc;
    // greedy-fallback reach list, refreshed with choice_info (xe = 0: none)
    int32_t xe;
    const int32_t *xl32;  // [n][xe] the xe nearest nodes of each row, (d, id) order
    uint2 *xlw;           // [n][xe] {float bits of choice_info, node}
    uint2 *xxw;           // [n][REACH_EXTRA] up to REACH_EXTRA such nodes with tau > tau_min
    int32_t *xxn;         // [n] how many are stored (0: the list is unused)
    int32_t *xhot;        // [n] nodes above tau_min outside the list at the last pass
    float *xlb;           // [n] max choice_info over the other nodes j != i with eta^beta_ij at
                          // most that of the last listed node
    // far list (fe = 0: none): xf16 [n][fp], the fp = REACH_MAX + fe nearest nodes
    // of each row in (d, id) order; xfb [n] max choice_info over the nodes j != i
    // with eta^beta_ij at most that of the row's last far node
    int32_t fe, fp;
    const uint16_t *xf16;
    float *xfb;
    const uint32_t *skip; // nullptr, or a device flag: when set the pass does nothing
};

// Message returned by mmas_last_error(NULL) on the calling thread.
void set_thread_error(const std::string &msg);

// Every device allocation of a colony, a batch or a learned prior: cudaMalloc,
// or cudaErrorMemoryAllocation when mmas_debug_fail_allocation armed a failure.
cudaError_t device_malloc(void **p, size_t bytes);
template <typename T>
inline cudaError_t device_malloc(T **p, size_t bytes)
{
    return device_malloc(reinterpret_cast<void **>(p), bytes);
}

// ---------------------------------------------------------------------------
// Host launchers (return the launch's cudaError_t)
// ---------------------------------------------------------------------------
cudaError_t launch_distances(const int2 *xy, int32_t n, int32_t ld, int32_t *d, int *maxd,
                             cudaStream_t s);
cudaError_t launch_max_dist(const int32_t *d, int32_t n, int32_t ld, int *maxd, cudaStream_t s);
// eta^beta of every cell; with `table` (maxd + 1 floats, maxd >= every
// distance) through a table of the distance values, else cell by cell.
cudaError_t launch_eta_beta(const int32_t *d, int32_t n, int32_t ld, double beta, float *eb,
                            float *table, int32_t maxd, cudaStream_t s);
// Largest distance for which eta^beta goes through a table (16 MB).
constexpr int32_t ETA_TABLE_MAX = 1 << 22;
cudaError_t launch_candidates(const int32_t *d, int32_t n, int32_t ld, int32_t cl,
                              int32_t *cand32, uint16_t *cand16, cudaStream_t s);
cudaError_t launch_nn_tour(const int32_t *d, int32_t n, int32_t ld, int32_t *tour, Scalars *sc,
                           const void *list, bool list16, int L, int P, cudaStream_t s);
cudaError_t launch_init_colony(int32_t n, int32_t ld, double rho, double p_root, float *tau,
                               Scalars *sc, cudaStream_t s);

// Testing aid: make every staging wait of the construction kernels on the
// current device run out (ERR_STAGE_TIMEOUT) or behave normally again.
cudaError_t set_stage_wait_expiry(bool on);
cudaError_t plan_construct(const ConstructArgs &a, int num_sms, size_t smem_optin,
                           ConstructPlan *plan);
cudaError_t launch_construct(const ConstructArgs &a, const ConstructPlan &plan, cudaStream_t s);
// narrow: every colony has n <= 2048 (up to 16 warps per SM, else 12)
cudaError_t prepare_construct_batch(size_t smem_bytes, bool narrow);
cudaError_t launch_construct_batch(const ConstructArgs *args, const BatchChunk *chunks, int nchunks,
                                   unsigned *counter, int grid, int warps, size_t smem_bytes,
                                   bool narrow, cudaStream_t s);

cudaError_t launch_best(const BestArgs &a, cudaStream_t s);
cudaError_t launch_score(const ScoreArgs &a, int num_sms, cudaStream_t s);
cudaError_t launch_update(const UpdateArgs &a, int num_sms, cudaStream_t s);
cudaError_t launch_score_batch(const ScoreArgs *args, const int32_t *ant_colony, const int32_t *ant_base,
                               int total_ants, bool xy, cudaStream_t s);
cudaError_t launch_update_batch(const UpdateArgs *args, const int32_t *row_colony, const int32_t *row_base,
                                int total_rows, bool alpha1, cudaStream_t s);

}  // namespace mmas
