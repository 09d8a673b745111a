/*
 * mmas.h -- C ABI of the GB300 MAX-MIN Ant System library (libmmas.so).
 *
 * The library runs the data-parallel hot path of the MAX-MIN Ant System for
 * the symmetric TSP (Skinderowicz, "Implementing a GPU-based parallel MAX-MIN
 * Ant System", FGCS 2020) on one NVIDIA GPU (sm_103a):
 *   - solution construction by m ants (Alg. 1, inner loops), with candidate
 *     lists (Sec. 4.3), a bitmask tabu (Sec. 4.1) and weighted reservoir
 *     sampling of Eq. (1) (Alg. 4, logarithmic keys of Sec. 4.2.2);
 *   - tour lengths, iteration best, global best and trail limits (Alg. 1);
 *   - evaporation, deposit and clamping to [tau_min, tau_max] (Sec. 2.1),
 *     fused with the refresh of choice_info (Sec. 2.1, Sec. 4.2.2).
 *
 * Conventions for every call:
 *   - Pointers named in a call are HOST pointers unless stated otherwise; the
 *     library copies what it needs and never keeps a caller pointer.
 *   - Every call returns an mmas_status.  On failure the handle is left as it
 *     was before the call and mmas_last_error() describes the failure.
 *   - A handle is not thread-safe; use one handle per thread.
 *   - mmas_iterate() and the other enqueueing calls are asynchronous on the
 *     handle's stream; errors raised on the device (a timed-out wait, an
 *     inconsistent state) surface at the next synchronising call.
 *   - Results are deterministic: (instance, params, seed, iteration count)
 *     fixes every tour, independent of launch shapes, because every random
 *     draw is keyed by (seed, iteration, ant, step, slot) -- see mmas_params.
 */
#ifndef MMAS_H
#define MMAS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MMAS_OK = 0,
    MMAS_EINVAL = 1,    /* a parameter or instance value is out of range     */
    MMAS_ENOMEM = 2,    /* a device or host allocation failed                */
    MMAS_ECUDA = 3,     /* a CUDA runtime call failed                        */
    MMAS_EOVERFLOW = 4, /* n * max(d) does not fit a 32-bit tour length      */
    MMAS_ETIMEOUT = 5,  /* a bounded device-side wait expired                */
    MMAS_ESTATE = 6     /* the call does not fit the handle's state          */
} mmas_status;

/* A symmetric TSP instance on n cities (Sec. 2.1).  Exactly one of xy and
 * dist is non-NULL.
 *   xy   : host, n x 2 int32 coordinates (row-major).  Distances are the
 *          TSPLIB rounded Euclidean nint(sqrt(dx^2 + dy^2)), computed exactly
 *          in integers.  |x|, |y| < 2^30.
 *   dist : host, n x n int32 distances, row-major, symmetric, >= 0, zero
 *          diagonal.
 * 3 <= n <= 65535 (node ids fit 16 bits, as in the paper's Table 1). */
typedef struct {
    int32_t n;
    const int32_t *xy;
    const int32_t *dist;
} mmas_instance;

/* Parameters.  mmas_default_params() fills the defaults shown.
 *   m        ants per iteration, 1 <= m <= 1048576                 (n)
 *   alpha    pheromone exponent of Eq. (1), >= 0                   (1)
 *   beta     heuristic exponent of Eq. (1), >= 0                   (2)
 *   rho      evaporation RATE: tau <- max((1 - rho) tau, tau_min), 0 < rho < 1.
 *            The paper's rho is the persistence (its rho = 0.5 is rho = 0.5
 *            here, its rho = 0.9 is rho = 0.1 here).                (0.02)
 *   p_best   the Stuetzle-Hoos parameter fixing tau_min/tau_max, 0 < p_best < 1
 *                                                                   (0.01)
 *   cl       candidate-list length: 0 samples the whole row (Eq. (1) over all
 *            unvisited nodes); 1..64 samples the cl nearest nodes (Sec. 4.3),
 *            cl < n.  Up to 32 one warp lane scores one candidate; above 32
 *            each lane scores two (slots l and l + 32).  ls needs cl <= 32 (32)
 *   seed     key of the counter-based generator (Philox4x32-10)    (1)
 *   deposit  0: deposit on the iteration best, 1: on the global best (0)
 *   fallback when every candidate of the current node is visited:
 *            0: take the unvisited node of largest choice_info (ties -> lower id);
 *            1: reservoir-sample all unvisited nodes                (0)
 *   device   CUDA device ordinal                                   (0)
 *   ant_offset  global index of this colony's first ant: a colony sharded
 *            over ranks gives each rank ants [ant_offset, ant_offset + m) of
 *            the whole colony, and the draws are keyed by the global index, so
 *            the union of the shards builds the same tours as one colony (0)
 *   ls       local search after construction (Sec. 5.7): 0 none; 1 2-opt the
 *            iteration best; 2 2-opt every ant's tour.  Bentley's 2-opt with
 *            the candidate lists as neighbour lists and don't-look bits, first
 *            improvement, cities visited in index order, runs repeated until
 *            one makes no move.  Needs cl >= 1 and 12.125n bytes + 2.25 KB
 *            of shared memory per CTA (n <= 18,979 on GB300)          (0)
 *   selection  whole-row mode (cl = 0) only: 0 weighted reservoir sampling
 *            (Alg. 4); 1 the parallel roulette wheel (Sec. 4.2.1), one draw
 *            per step, the exact single-precision procedure described below (0)
 *   tabu     whole-row mode only: 0 the bitmask tabu; 1 the compact list of
 *            unvisited nodes (Sec. 4.1): removing the node at slot j moves the
 *            list's last node into slot j                           (0)
 *   stream   cudaStream_t to enqueue on, or NULL for a private non-blocking
 *            stream; pass cudaStreamLegacy to use the legacy default stream (NULL)
 *
 * Random draws (k = ant_offset + local ant index): start node of ant k in iteration it = word 0 of
 * Philox(ctr = (0xFFFFFFFF, 0, k, it)); candidate slot s at step t = word
 * (t mod 4) of Philox(ctr = (s, t/4, k, it)); whole-row node v at step t =
 * word (v mod 4) of Philox(ctr = (2^31 | v/4, t, k, it)); key = (seed_lo,
 * seed_hi).  A word x maps to r = ((x >> 9) + 1/2) 2^-23 in (0,1).
 * Compact-list reservoir draws: slot j at step t = word (j mod 4) of
 * Philox(ctr = (2^30 | j/4, t, k, it)).  Roulette wheel: one draw per step,
 * word 0 of Philox(ctr = (0xFFFFFFFE, t, k, it)), u = r in single precision.
 * The roulette wheel takes the unvisited weights (choice_info) in node order
 * (bitmask tabu, visited nodes at weight 0) or list order (compact tabu), in
 * rounds of 128 positions: lane l of 32 owns positions 128r + 4l .. +3 and
 * forms partial sums q0 = x0, q1 = q0 + x1, q2 = q1 + x2, q3 = q2 + x3; the
 * lanes' q3 are scanned (for d = 1, 2, 4, 8, 16: S_l += S_{l-d} when l >= d)
 * and the rounds' totals S_31 accumulate into the offset O; with T = the
 * final O and theta = u T, the pick is the first position p with x_p > 0 and
 * (O_r + S_{l-1}) + q_e > theta (S_{-1} = 0), else the last p with x_p > 0;
 * every operation is a float add or multiply rounded to nearest. */
typedef struct {
    int32_t m;
    float alpha;
    float beta;
    float rho;
    float p_best;
    int32_t cl;
    uint64_t seed;
    int32_t deposit;
    int32_t fallback;
    int32_t device;
    int32_t ant_offset;
    int32_t ls;
    int32_t selection;
    int32_t tabu;
    void *stream;
} mmas_params;

typedef struct mmas_handle mmas_handle;

/* Counters and launch facts of a handle (filled by mmas_stats). */
typedef struct {
    int64_t iterations;        /* completed iterations (the next iteration's index)  */
    int64_t fallback_steps;    /* candidate-list fallbacks since create              */
    int64_t nn_len;            /* nearest-neighbour tour length (initial limits)     */
    int32_t best_len;          /* global best length, -1 before the first iteration  */
    int32_t iter_best_len;     /* last iteration best, -1 before the first iteration */
    float tau_min, tau_max;    /* current trail limits                               */
    int32_t construct_grid;    /* CTAs of the construction kernel                    */
    int32_t construct_block;   /* threads per CTA (one warp per ant)                 */
    int32_t construct_staged;  /* 1 if the choice table is staged in shared memory   */
    int32_t construct_smem;    /* dynamic shared memory per CTA, bytes               */
    int32_t row_pitch;         /* elements per row of the n x n device matrices      */
    int64_t fallback_scans;    /* of the fallback steps, those that scanned the row
                                  (the rest were decided on the nearest nodes' lists:
                                  the 128 nearest, and above 8,192 nodes the 1024
                                  nearest)                                          */
} mmas_stats_t;

/* Fill *p with the defaults listed at mmas_params (m = 0 means "m = n"). */
void mmas_default_params(mmas_params *p);

/* Build a colony (Alg. 1 before the main loop, Sec. 2.1, Sec. 4.3): copy the
 * instance to the device, compute distances, eta^beta = d^-beta (d clamped to
 * >= 1), candidate lists ordered by (distance, id), the nearest-neighbour tour
 * from node 0, tau_max = 1/(rho C_nn), tau_min = tau_max (1 - p)/((n/2 - 1) p)
 * with p = p_best^(1/n), tau <- tau_max and choice_info.  Returns the handle
 * in *out (NULL on failure).  Errors: EINVAL (bad value; message says which),
 * EOVERFLOW (n * max d >= 2^31), ENOMEM, ECUDA.  Synchronises the stream. */
mmas_status mmas_create(const mmas_instance *inst, const mmas_params *p, mmas_handle **out);

/* Enqueue k >= 0 iterations of Alg. 1's main loop (construction, tour
 * lengths, iteration best, global best and limits, evaporation, deposit,
 * choice_info refresh), replayed from one CUDA graph per iteration.  No host
 * synchronisation.  Errors: EINVAL (k < 0), ESTATE, ECUDA. */
mmas_status mmas_iterate(mmas_handle *h, int32_t k);

/* Synchronise, then copy the global-best tour (n ids) to tour_out (may be
 * NULL) and its length to *len_out (may be NULL).  Errors: ESTATE before the
 * first iteration, ETIMEOUT / ESTATE if a device-side check failed. */
mmas_status mmas_best_tour(mmas_handle *h, int32_t *tour_out, int32_t *len_out);

/* Free every resource of the handle (NULL is allowed). */
void mmas_destroy(mmas_handle *h);

/* Message of the last failed call on h, or of the calling thread's last
 * failed mmas_create when h is NULL.  Never NULL; "" when nothing failed. */
const char *mmas_last_error(const mmas_handle *h);

/* ---- lower-level steps and state access (tests, benchmarks, resume) ---- */

/* Enqueue construction only (Alg. 1 inner loops and the tour lengths) for the
 * current iteration index, leaving pheromone, limits and the index as they
 * are.  The tours are readable with mmas_get_tours. */
mmas_status mmas_construct(mmas_handle *h);

/* Enqueue the rest of one iteration with a caller-given tour (host, n ids, a
 * permutation) of length len standing in for the iteration best: global best
 * and limits (Alg. 1), evaporation, deposit, choice_info.  The iteration index
 * is not advanced.  Errors: EINVAL (not a permutation, len <= 0). */
mmas_status mmas_update(mmas_handle *h, const int32_t *tour, int32_t len);

/* ---- one colony sharded over ranks: the exchange on device buffers -------
 *
 * Ants are independent given the pheromone (Sec. 2.1), so rank r can build
 * ants [ant_offset, ant_offset + m) of a colony of M ants (mmas_params.m = the
 * rank's count, ant_offset its first global index; draws are keyed by the
 * global index).  Alg. 1's iteration best over all ranks then takes, per
 * iteration, after mmas_construct on every rank:
 *   mmas_shard_best_key      -> all-reduce (MIN) of the 8-byte key,
 *   mmas_shard_tour          -> all-reduce (SUM) of the n-int tour buffer,
 *   mmas_update_device       (the same update on every replica),
 * e.g. with NCCL on the colony's stream: 8 + 4n bytes per rank, no host copy.
 * All three are enqueued on the colony's stream; pointers are DEVICE pointers
 * on the colony's device.  Errors: EINVAL (NULL pointer), ECUDA. */

/* *d_key (1 int64) = (L << 32) | (ant_offset + k) for the shortest tour k of
 * the last construction (ties -> lower k): the all-reduced MIN of the ranks'
 * keys is Alg. 1's iteration best over the whole colony. */
mmas_status mmas_shard_best_key(mmas_handle *h, int64_t *d_key);

/* d_tour (n int32) = the tour of global ant (*d_key & 0xFFFFFFFF) when this
 * rank builds that ant, else n zeros: the element-wise SUM over the ranks is
 * that tour on every rank. */
mmas_status mmas_shard_tour(mmas_handle *h, const int64_t *d_key, int32_t *d_tour);

/* mmas_update with a device-side tour d_tour (n int32) and length
 * (*d_key >> 32): global best and limits, evaporation, deposit, choice_info;
 * then the iteration index advances, as after a whole iteration, so that
 * construct, exchange and update repeat with no host call in between.  The
 * tour is checked on the device; if
 * it is not a permutation of 0..n-1 (or the length is not positive) the update
 * does nothing and the next synchronising call returns MMAS_ESTATE. */
mmas_status mmas_update_device(mmas_handle *h, const int32_t *d_tour, const int64_t *d_key);

/* The colony's 2-opt (Sec. 5.7, as ls applies it: the candidate lists as
 * neighbour lists, don't-look bits, first improvement until no move) applied
 * to a caller's tour: `tour` (host, n ids, a permutation) is improved in place
 * and its length written to *len_out (may be NULL).  The colony's state is not
 * changed.  Needs 1 <= cl <= 32; the first call on a colony created without
 * local search computes its neighbour distances.  Synchronises.  Errors:
 * EINVAL (not a permutation, cl, n too large), ESTATE (move cap), ECUDA. */
mmas_status mmas_two_opt_tour(mmas_handle *h, int32_t *tour, int32_t *len_out);

/* Synchronise and copy the last constructed tours (m x n, row-major) and
 * their lengths (m).  Either pointer may be NULL. */
mmas_status mmas_get_tours(mmas_handle *h, int32_t *tours, int32_t *lens);

/* Synchronise and copy the pheromone matrix (n x n, row-major) and the
 * current limits.  Any pointer may be NULL. */
mmas_status mmas_get_pheromone(mmas_handle *h, float *tau, float *tau_min, float *tau_max);

/* Replace the pheromone matrix (n x n, row-major, finite, > 0) and the limits
 * (0 < tau_min <= tau_max), then refresh choice_info.  Enqueued. */
mmas_status mmas_set_pheromone(mmas_handle *h, const float *tau, float tau_min, float tau_max);

/* Synchronise and copy the set-up results: distances (n x n), eta^beta
 * (n x n), candidate lists (n x cl) and the nearest-neighbour length.  Any
 * pointer may be NULL. */
mmas_status mmas_get_setup(mmas_handle *h, int32_t *dist, float *eta_beta, int32_t *cand,
                           int64_t *nn_len);

/* Set the iteration index used by the random draws of the next construction
 * (for resuming a run, and for repeated draws under a fixed pheromone). */
mmas_status mmas_set_iteration(mmas_handle *h, int32_t it);

/* Synchronise and fill *out. */
mmas_status mmas_stats(mmas_handle *h, mmas_stats_t *out);

/* Testing aid for the out-of-memory paths (not part of the method): arm a
 * failure of the device allocation `after` allocations from now (0: the next
 * one) made by mmas_create, mmas_batch_create, the learned prior's calls and
 * the calls they make; that allocation fails as if the device were out of
 * memory, the call returns MMAS_ENOMEM and frees what it had allocated, and
 * the arming is spent.  after < 0 disarms.  Process-wide. */
void mmas_debug_fail_allocation(int32_t after);

/* Testing aid for the bounded device waits (not part of the method): with
 * on != 0, every construction launch on `device` that stages its table in
 * shared memory first waits for a flag that nothing sets, gives up after its
 * 1 ms limit, lets its own bulk copies land (bounded, 2 s), records a timeout
 * and leaves without building tours; the next synchronising call on the
 * colony reports MMAS_ETIMEOUT and the colony's results are void.  on = 0
 * restores normal waits.  Errors: EINVAL (bad device), ECUDA. */
mmas_status mmas_debug_expire_stage_waits(int32_t device, int32_t on);

/* Testing aid for the 2-opt search's guard (not part of the method): every
 * improving move shortens the tour, so a search ends by itself; a cap of 64 n
 * moves per tour only guards against a defect.  cap > 0 replaces it on
 * `device` (a search that reaches it stops, keeps the moves made, and the next
 * synchronising call returns MMAS_ESTATE); cap <= 0 restores 64 n.
 * Errors: EINVAL (bad device), ECUDA. */
mmas_status mmas_debug_two_opt_move_cap(int32_t device, int64_t cap);

/* Block until all work enqueued by the handle has finished; report device-side
 * errors (ETIMEOUT, ESTATE) raised since the last check. */
mmas_status mmas_synchronize(mmas_handle *h);

/* Phase timing (a measurement aid; the paper times its kernels with CUDA
 * timers, Sec. 5).  enable != 0 re-records the iteration graph with CUDA
 * event-record nodes before construction, after construction and after the
 * pheromone pass; enable == 0 records it without them. */
mmas_status mmas_enable_phase_timing(mmas_handle *h, int32_t enable);

/* Synchronise and report the phase durations of the most recent iteration run
 * by mmas_iterate with phase timing enabled, in milliseconds: construction
 * (incl. tour lengths), the rest (best, limits, pheromone pass), and the whole
 * iteration.  Any pointer may be NULL.  ESTATE if timing is not enabled or no
 * timed iteration has run. */
mmas_status mmas_phase_times(mmas_handle *h, float *construct_ms, float *rest_ms, float *total_ms);

/* Measurement aid (not part of the method): the arithmetic ceiling of one
 * selection on device `device`.  Runs only the per-candidate work of a
 * candidate-list step (Alg. 4 with log keys, Sec. 4.2.2) -- one Philox4x32-10
 * output word, its (0,1) uniform, log2, the key multiply and a running maximum
 * -- at full occupancy for about ms milliseconds, and writes the rate in draws
 * per second to *draws_per_s.  Synchronous; allocates and frees a small device
 * buffer.  Errors: EINVAL (NULL output, ms <= 0), ECUDA. */
mmas_status mmas_probe_draw_rate(int32_t device, float ms, double *draws_per_s);

/* Measurement aid (not part of the method): the L2 read bandwidth of device
 * `device`, the ceiling for bytes that a kernel finds in L2 rather than in
 * HBM.  A read-only kernel sweeps a `bytes`-byte buffer (small enough to stay
 * resident in L2: 16-64 MiB on GB300) with 16-byte loads that bypass L1, many
 * passes per launch at full occupancy; *gbs = the best of 10 launches in
 * GB/s (10^9 bytes read per second).  Synchronous; allocates and frees the
 * buffer.  Errors: EINVAL (NULL gbs, bytes outside [1 MiB, 1 GiB]), ENOMEM,
 * ECUDA. */
mmas_status mmas_probe_l2_bandwidth(int32_t device, int64_t bytes, double *gbs);

/* Test hook (not part of the method): the accuracy of the log2 the
 * candidate-list steps take of their draws (the reservoir key log2(r)/w,
 * Sec. 4.2.2).  Evaluates it on device `device` at every one of the 2^23 draw
 * values r = ((x >> 9) + 1/2) 2^-23 and writes the largest relative error
 * against the double-precision log2 to *max_rel, and that of the library's
 * log2f to *max_rel_library (may be NULL).  Synchronous; allocates and frees a
 * 16-byte device buffer.  Errors: EINVAL (NULL max_rel), ECUDA. */
mmas_status mmas_debug_draw_log2_error(int32_t device, double *max_rel, double *max_rel_library);

/* ---- learned edge prior: tensor-core GEMM ---------------------------------
 *
 * BF16 GEMM on the tensor cores (tcgen05, FP32 accumulation in tensor memory),
 * the dense contraction of the learned edge prior (a message-passing network
 * over the candidate-list graph; not in the paper):
 *   out[m][j] = act( sum_k A[m][k] * B[j][k] + bias[j] ),  0 <= j < n
 *   d_a   device bf16, m rows of k values, row stride lda >= k (elements)
 *   d_b   device bf16, n rows of k values, row stride ldb >= k
 *   d_bias device fp32 [n] or NULL;  relu != 0 applies max(x, 0)
 *   d_out device fp32, m rows, row stride ldd >= n
 *   1 <= n <= 128 (tiles of 64 or 128 columns), m >= 0, k >= 0 arbitrary.
 * Synchronises `stream` (a cudaStream_t, NULL: legacy) before returning.
 * Errors: EINVAL (message in mmas_last_error(NULL)), ECUDA, ETIMEOUT (an MMA
 * did not complete within 2 s). */
mmas_status mmas_gemm_bf16(const void *d_a, int32_t lda, const void *d_b, int32_t ldb,
                           const float *d_bias, float *d_out, int32_t ldd, int32_t m, int32_t n,
                           int32_t k, int32_t relu, void *stream);

/* The same product accumulated, for long K (the weight gradients of the
 * learned prior, K = n):  out[m][j] += sum_k A[m][k] * B[j][k].  The K blocks
 * (64 wide) are split over CTAs, up to one per SM, each adding its partial
 * 128 x n tile into d_out with fp32 atomic adds, so the order of the additions
 * (and the last bits of the result) may vary between calls.  Arguments and
 * errors as for mmas_gemm_bf16 (no bias or activation). */
mmas_status mmas_gemm_bf16_acc(const void *d_a, int32_t lda, const void *d_b, int32_t ldb, float *d_out,
                               int32_t ldd, int32_t m, int32_t n, int32_t k, void *stream);

/* ---- learned edge prior ---------------------------------------------------
 *
 * A 3-layer message-passing network over each node's 16 nearest neighbours
 * (the first 16 entries of a colony's candidate lists, so cl >= 16; the
 * instance must have coordinates) scores every candidate edge; its edge
 * probabilities sigmoid(s) replace eta^beta in that colony's choice_info (an
 * extension of this library; plain MMAS with eta = 1/d stays available and is
 * the reference).  Hidden width 64; every dense product runs on the tensor
 * cores (bf16 operands, fp32 accumulation).
 *   features  F0[i] = ((x-cx)/s, (y-cy)/s, d(i,nn0)/D, d(i,nn1)/D, d(i,nn3)/D,
 *             d(i,nn15)/D, 1, 0): (cx, cy) the centre of the coordinates'
 *             bounding box, s its longer side, D = max_i d(i, nn[i][15])
 *   h0 = relu(F0 W0^T + b0);  for l = 1..3: m_i = mean_k h[nn[i][k]],
 *   h = relu([h | m] W_l^T + b_l) + h;  q = h Wq^T;
 *   s[i][k] = <q_i, h[nn[i][k]]> / 8 + a d(i,nn[i][k])/D + c
 * Parameters, fp32, in this order: W0 [64][8], b0 [64], W1 [64][128], b1 [64],
 * W2, b2, W3, b3, Wq [64][64], a, c  (MMAS_PRIOR_PARAMS values; weights
 * row-major [out][in]).  Every call enqueues on the colony's stream and
 * synchronises it before returning.  Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
typedef struct mmas_prior mmas_prior;
#define MMAS_PRIOR_PARAMS 29442

/* params: host, MMAS_PRIOR_PARAMS floats, or NULL for zeros. */
mmas_status mmas_prior_create(const float *params, int32_t device, mmas_prior **out);
/* Replace the parameters (and reset the optimiser state). */
mmas_status mmas_prior_set_params(mmas_prior *p, const float *params);
mmas_status mmas_prior_get_params(mmas_prior *p, float *params);
/* The optimiser's state, for checkpoints and for checking a training step:
 * Adam's first and second moments m and v (host, MMAS_PRIOR_PARAMS floats
 * each), the gradient computed by the last mmas_prior_train step or
 * mmas_prior_grad call (host, MMAS_PRIOR_PARAMS floats; zeros before any), and
 * the number of Adam steps taken (*step).  Any pointer may be NULL.
 * Synchronises the device. */
mmas_status mmas_prior_get_state(mmas_prior *p, float *m, float *v, float *grad, int32_t *step);
/* Restore Adam's moments (finite, v >= 0) and step count, e.g. from a
 * checkpoint written with mmas_prior_get_state.  Errors: EINVAL. */
mmas_status mmas_prior_set_state(mmas_prior *p, const float *m, const float *v, int32_t step);
/* Scores s [n][16] (host, row-major) of colony h's candidate edges. */
mmas_status mmas_prior_scores(mmas_prior *p, mmas_handle *h, float *scores);
/* `steps` Adam steps (Kingma and Ba, "Adam: a method for stochastic
 * optimization", ICLR 2015; lr; beta1 0.9, beta2 0.999, eps 1e-8, each a
 * single-precision value; per parameter m <- b1 m + (1 - b1) g,
 * v <- b2 v + (1 - b2) g^2, theta <- theta - lr (m / c1) / (sqrt(v / c2) + eps)
 * with c1 = 1 - b1^t, c2 = 1 - b2^t for step number t) on the mean binary
 * cross-entropy of sigmoid(s) against y[i][k] = [(i, nn[i][k]) is an edge of
 * `tour`] (host, a permutation of 0..n-1); *loss (may be NULL) = the loss of
 * the last step's forward pass. */
mmas_status mmas_prior_train(mmas_prior *p, mmas_handle *h, const int32_t *tour, int32_t steps, float lr,
                             float *loss);
/* The gradient of that loss at the current parameters (host, MMAS_PRIOR_PARAMS
 * floats) without changing the parameters or the optimiser state. */
mmas_status mmas_prior_grad(mmas_prior *p, mmas_handle *h, const int32_t *tour, float *grad, float *loss);
/* Replace colony h's eta^beta: the 16 candidates of row i take sigmoid(s[i][k]);
 * every other entry keeps d^-beta scaled by min_k sigmoid(s[i][k]) / (the 16th
 * candidate's d^-beta).  Then choice_info is refreshed from the current
 * pheromone.  The colony's pheromone, limits and iteration index are unchanged. */
mmas_status mmas_prior_apply(mmas_prior *p, mmas_handle *h);
/* Weight instead of replace: eta^beta of the 16 candidate edges of row i is
 * multiplied by sigmoid(s[i][k])^gamma, every other entry of the row by
 * (min_k sigmoid(s[i][k]))^gamma; gamma = 0 leaves plain MMAS, 0 <= gamma <= 64.
 * Then choice_info is refreshed as by mmas_prior_apply.  Errors as there. */
mmas_status mmas_prior_apply_weighted(mmas_prior *p, mmas_handle *h, float gamma);
void mmas_prior_destroy(mmas_prior *p);
const char *mmas_prior_last_error(const mmas_prior *p);

/* ---- batched colonies -----------------------------------------------------
 *
 * Many independent colonies, on instances of uneven size, advanced together.
 * Every iteration (Alg. 1) of all of them is three launches, recorded once as
 * a CUDA graph: one persistent construction launch that hands (colony, group of
 * ants) chunks to CTAs from a global counter, largest colonies first, staging
 * each colony's candidate table in shared memory when it fits; one scoring
 * launch (lengths, then each colony's iteration best, global best and limits);
 * one fused pheromone launch over the rows of every colony.
 *
 * Colony b is exactly the colony mmas_create would build from instances[b]
 * with the shared params, except seed = params.seed + b and m = params.m (n_b
 * when params.m is 0): same tours, lengths and pheromone, iteration by
 * iteration, whatever the launch configuration.  Restrictions: 1 <= cl <= 32
 * (candidate lists), ls = 0, ant_offset = 0; either every instance has
 * coordinates or every instance has a matrix.  count >= 1.  The batch
 * enqueues on params.stream (NULL: a private non-blocking stream).
 * Errors: EINVAL (a restriction or an instance's validation fails; the message
 * names the colony), ENOMEM, ECUDA; on error nothing is created. */
typedef struct mmas_batch mmas_batch;

/* Launch shape of the batched construction: warps (= ants) per CTA and CTAs
 * per SM, 1..4 (shared memory per CTA is the SM's share); warps per CTA times
 * CTAs per SM is at most 16 when every colony has n <= 2048, else at most 12
 * (the registers of an SM).  The default is 16 (or 12) warps, one CTA per SM.
 * Results do not depend on it. */
typedef struct {
    int32_t warps_per_cta;
    int32_t ctas_per_sm;
} mmas_batch_config;

mmas_status mmas_batch_create(const mmas_instance *instances, int32_t count,
                              const mmas_params *params, mmas_batch **out);

/* Enqueue k iterations of every colony (k >= 0). */
mmas_status mmas_batch_iterate(mmas_batch *b, int32_t k);

/* Synchronise; copy colony c's global best tour (n_c ids) and length.  ESTATE
 * before the first iteration.  Either pointer may be NULL. */
mmas_status mmas_batch_best_tour(mmas_batch *b, int32_t colony, int32_t *tour_out,
                                 int32_t *len_out);

/* Synchronise; copy every colony's global best length (count int32, -1 before
 * the first iteration) in one transfer. */
mmas_status mmas_batch_best_lengths(mmas_batch *b, int32_t *lens_out);

/* Synchronise; copy colony c's last tours (m_c x n_c) and lengths (m_c).
 * Either pointer may be NULL. */
mmas_status mmas_batch_get_tours(mmas_batch *b, int32_t colony, int32_t *tours, int32_t *lens);

/* Colony c as an ordinary handle (*out), owned by the batch: valid until
 * mmas_batch_destroy and never passed to mmas_destroy.  Every other call that
 * takes a handle accepts it (a learned prior trains on and applies to it, for
 * instance); batch iterations and calls on the handle advance the same colony.
 * Errors: EINVAL (bad colony index, NULL out). */
mmas_status mmas_batch_colony(mmas_batch *b, int32_t colony, mmas_handle **out);

/* Use launch shape *cfg for the construction (re-records the graph). */
mmas_status mmas_batch_set_config(mmas_batch *b, const mmas_batch_config *cfg);
mmas_status mmas_batch_get_config(mmas_batch *b, mmas_batch_config *cfg);

/* Autotuner: time the construction launch under each candidate launch shape
 * (reps launches each, median; the colonies' pheromone and iteration indices
 * are untouched and the tours are rebuilt by the next iteration), keep the
 * fastest and write it to *chosen (may be NULL).  Fallback counters are reset. */
mmas_status mmas_batch_autotune(mmas_batch *b, int32_t reps, mmas_batch_config *chosen);

/* Block until the batch's work is done; report device-side errors. */
mmas_status mmas_batch_synchronize(mmas_batch *b);

/* Phase timing as for one colony: construction vs. the rest, for the most
 * recent iteration run by mmas_batch_iterate with timing on. */
mmas_status mmas_batch_enable_phase_timing(mmas_batch *b, int32_t enable);
mmas_status mmas_batch_phase_times(mmas_batch *b, float *construct_ms, float *rest_ms,
                                   float *total_ms);

/* Sum of the colonies' fallback steps since creation (or the last autotune). */
mmas_status mmas_batch_fallback_steps(mmas_batch *b, int64_t *out);

void mmas_batch_destroy(mmas_batch *b);
const char *mmas_batch_last_error(const mmas_batch *b);

/* ---- allocation-free scoring ----------------------------------------------
 *
 * For callers that must not have a library allocate device memory: serving
 * loops that cannot afford cudaMalloc/cudaFree (they synchronise the whole
 * device and stall every other stream), and frameworks whose caching allocator
 * owns the device memory budget.  The paper has no counterpart; it is a service
 * of this library.
 *
 * mmas_score_tours_noalloc computes, for m tours already in device memory, the
 * length of each tour (TSPLIB rounded Euclidean distances, exact integers) and
 * the shortest one, exactly as the iteration-best step does, but with no
 * handle and without allocating: the caller passes every input and output, and
 * the only scratch is a fixed array inside the library (one 8-byte partial
 * minimum per CTA for at most 4,096 CTAs, plus a counter: about 33 KB per GPU,
 * held from library load until the process exits).
 *   d_tours  device, m x pitch int32; row k's first n entries are a tour (a
 *            permutation of 0..n-1)
 *   m        1 <= m <= MMAS_NOALLOC_MAX_ANTS
 *   n        3 <= n <= 65535;  pitch >= n (elements per row)
 *   d_xy     device, n x 2 int32 coordinates, |x|, |y| < 2^30, 8-byte aligned
 *            (the other buffers 4-byte aligned)
 *   d_lens   device, m int32 (out): tour lengths; n * max(d) must be < 2^31
 *   d_best   device, 2 int32 (out): {shortest length, lowest ant reaching it}
 *   stream   cudaStream_t to enqueue on (NULL: the legacy default stream)
 * Asynchronous: the results are ready when the stream reaches them.
 * Errors: EINVAL for a NULL buffer or a size out of range (checked before any
 * GPU work, message in mmas_last_error(NULL)); ECUDA if a CUDA call fails.
 * The first call on each device looks up the scratch's device address with
 * that device current and keeps it for the life of the process; make that
 * first call before any stream capture.  cudaDeviceReset unloads the library's
 * device code and so invalidates the kept address: after resetting a device,
 * do not call this entry point on it again in the same process.
 * Every call shares the scratch and a call leaves it holding its own partial
 * results, so calls whose GPU work may overlap (e.g. on different streams
 * with no ordering between them) race and must be serialised by the caller. */
#define MMAS_NOALLOC_MAX_ANTS 1048576
mmas_status mmas_score_tours_noalloc(const int32_t *d_tours, int32_t m, int32_t n, int32_t pitch,
                                     const int32_t *d_xy, int32_t *d_lens, int32_t *d_best,
                                     void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MMAS_H */
