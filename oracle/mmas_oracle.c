/*
 * CPU oracle for the MAX-MIN Ant System hot path (symmetric TSP).
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the
 * benchmark's CPU-baseline leg are the only callers.  The CUDA library never
 * calls, links or shares code with this file, and the oracle does not read
 * anything the CUDA library produced.
 *
 * It restates, plainly and slowly, what Skinderowicz, "Implementing a
 * GPU-based parallel MAX-MIN Ant System" (FGCS 2020) computes:
 *   - the problem and the heuristic information (Sec. 2.1);
 *   - the selection probabilities of Eq. (1), sampled by weighted reservoir
 *     sampling (Alg. 3, Alg. 4) with the logarithmic key of Sec. 4.2.2;
 *   - candidate lists (Sec. 4.3);
 *   - the MMAS main loop, Alg. 1: construction, iteration best, global best
 *     and trail limits, evaporation, deposit (Sec. 2.1, Sec. 4.4).
 *
 * Floating point is double precision, except that the pheromone, the
 * heuristic weights eta^beta and choice_info are stored as 32-bit floats
 * (the paper's storage type, Sec. 4.2.2) and rounded to float where they are
 * stored.  No step is blocked, fused or reordered.
 *
 * Readings taken where the paper is silent (each repeated at its function):
 *   R-rho   the parameter rho is the evaporation rate: tau <- (1-rho) tau,
 *           and (1-rho) is held as a float, like the pheromone it scales;
 *   R-lim   tau_max = 1/(rho C), tau_min = tau_max (1-p)/((n/2 - 1) p),
 *           p = p_best^(1/n), following Stuetzle and Hoos (2000);
 *   R-dep   deposit on both (i,j) and (j,i); Delta = 1/C rounded to float;
 *   R-bound every trail stays in [tau_min, tau_max]: evaporation clamps both
 *           ways (the cap matters only when tau_max drops, see orc_evaporate);
 *   R-eta   eta^beta = d^-beta with d clamped to >= 1; zero on the diagonal;
 *   R-fb    when every candidate is visited, pick the unvisited node with the
 *           largest choice_info (ties -> lower id), or, with fallback = 1,
 *           sample all unvisited nodes by the same reservoir rule;
 *   R-rng   Philox4x32-10 counters (see orc_word_* below);
 *   R-tie   ties go to the lower node id, the lower ant index, and the
 *           global best is replaced only by a strictly shorter tour;
 *   R-nint  d = nint(sqrt(dx^2 + dy^2)), computed exactly in integers.
 *
 * Parity: every function here is pinned by the CPU tests (known-answer
 * vectors, closed forms, brute force, invariants, chi-square).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers (reading R-rng)                             */
/* ------------------------------------------------------------------------ */

/* Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11): ten rounds; each round takes
 * two 32x32->64 products of counter words 0 and 2 with the round multipliers,
 * and the key is bumped by the Weyl constants between rounds. */
ORC_API void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void philox_seeded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Map a 32-bit word to the open interval (0,1): ((x >> 9) + 1/2) * 2^-23.
 * The 23 kept bits plus the half make every value exact in float and double. */
ORC_API double orc_uniform01(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Start node draw (Alg. 1: u <- U{0, n-1}): word 0 of the counter
 * (0xFFFFFFFF, 0, ant, iteration). */
ORC_API uint32_t orc_word_start(uint64_t seed, int32_t it, int32_t ant)
{
    uint32_t o[4];
    philox_seeded(seed, 0xFFFFFFFFu, 0u, (uint32_t)ant, (uint32_t)it, o);
    return o[0];
}

/* Uniform for candidate-list slot s at step t (Alg. 4 line "r <- random(0,1)"):
 * word (t mod 4) of the counter (s, floor(t/4), ant, iteration). */
ORC_API uint32_t orc_word_cand(uint64_t seed, int32_t it, int32_t ant, int32_t t, int32_t s)
{
    uint32_t o[4];
    philox_seeded(seed, (uint32_t)s, (uint32_t)t >> 2, (uint32_t)ant, (uint32_t)it, o);
    return o[t & 3];
}

/* Uniform for node v when the whole row is sampled (no candidate list, or
 * fallback = 1): word (v mod 4) of the counter (2^31 | floor(v/4), t, ant, it). */
ORC_API uint32_t orc_word_row(uint64_t seed, int32_t it, int32_t ant, int32_t t, int32_t v)
{
    uint32_t o[4];
    philox_seeded(seed, 0x80000000u | ((uint32_t)v >> 2), (uint32_t)t, (uint32_t)ant,
                  (uint32_t)it, o);
    return o[v & 3];
}

/* Whole-row variants (Sec. 4.1 compact tabu, Sec. 4.2.1 roulette wheel):
 * the reservoir draw of slot j of the compact list at step t, and the single
 * roulette-wheel draw of step t. */
ORC_API uint32_t orc_word_slot(uint64_t seed, int32_t it, int32_t ant, int32_t t, int32_t j)
{
    uint32_t o[4];
    philox_seeded(seed, 0x40000000u | ((uint32_t)j >> 2), (uint32_t)t, (uint32_t)ant,
                  (uint32_t)it, o);
    return o[j & 3];
}

ORC_API uint32_t orc_word_rwm(uint64_t seed, int32_t it, int32_t ant, int32_t t)
{
    uint32_t o[4];
    philox_seeded(seed, 0xFFFFFFFEu, (uint32_t)t, (uint32_t)ant, (uint32_t)it, o);
    return o[0];
}

/* floor(x * n / 2^32): the start node for a 32-bit word x. */
ORC_API int32_t orc_start_node(uint64_t seed, int32_t it, int32_t ant, int32_t n)
{
    uint64_t x = orc_word_start(seed, it, ant);
    return (int32_t)((x * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* The instance (Sec. 2.1)                                                  */
/* ------------------------------------------------------------------------ */

/* floor(sqrt(s)) by the bit-by-bit (digit-by-digit, base 2) method. */
ORC_API uint64_t orc_isqrt64(uint64_t s)
{
    uint64_t res = 0, bit = (uint64_t)1 << 62;
    while (bit > s) bit >>= 2;
    while (bit != 0) {
        if (s >= res + bit) {
            s -= res + bit;
            res = (res >> 1) + bit;
        } else {
            res >>= 1;
        }
        bit >>= 2;
    }
    return res;
}

/* Rounded Euclidean distance (reading R-nint): nint(sqrt(s)), s = dx^2 + dy^2.
 * With q = floor(sqrt(s)): sqrt(s) >= q + 1/2  <=>  s > q^2 + q, so
 * nint = q + [s > q^2 + q] (sqrt(s) is never exactly q + 1/2 for integer s). */
ORC_API int64_t orc_euc2d(int32_t x1, int32_t y1, int32_t x2, int32_t y2)
{
    int64_t dx = (int64_t)x1 - x2, dy = (int64_t)y1 - y2;
    uint64_t s = (uint64_t)(dx * dx) + (uint64_t)(dy * dy);
    uint64_t q = orc_isqrt64(s);
    return (int64_t)(q + (s > q * q + q ? 1 : 0));
}

/* Distance matrix d[i][j] (row-major n x n) from integer coordinates xy[i][2]. */
ORC_API void orc_distances(int32_t n, const int32_t *xy, int32_t *d)
{
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j)
            d[(size_t)i * n + j] = (int32_t)orc_euc2d(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1]);
}

/* Heuristic weights eta_ij^beta with eta_ij = 1/d_ij (Sec. 2.1), stored as
 * float; d is clamped to >= 1 inside eta only and the diagonal is 0 (R-eta). */
ORC_API void orc_eta_beta(int32_t n, const int32_t *d, double beta, float *eb)
{
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j) {
            if (i == j) { eb[(size_t)i * n + j] = 0.0f; continue; }
            int32_t dij = d[(size_t)i * n + j];
            double dd = dij < 1 ? 1.0 : (double)dij;
            eb[(size_t)i * n + j] = (float)pow(1.0 / dd, beta);
        }
}

/* Candidate lists (Sec. 4.3): for each node, the cl closest other nodes in
 * ascending (distance, id) order.  cand is n x cl.  Each row is one pass over
 * the other nodes j in increasing id, keeping the cl smallest (d, id) pairs
 * seen so far in order: a node enters when its distance is strictly smaller
 * than the last kept one's (an equal distance loses to the lower id already
 * kept), displacing the last. */
ORC_API void orc_candidates(int32_t n, const int32_t *d, int32_t cl, int32_t *cand)
{
    for (int32_t i = 0; i < n; ++i) {
        const int32_t *row = d + (size_t)i * n;
        int32_t *best = cand + (size_t)i * cl;
        int32_t k = 0;  /* entries kept so far */
        for (int32_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (k == cl && row[j] >= row[best[cl - 1]]) continue;
            int32_t p = k < cl ? k++ : cl - 1;  /* the slot j takes before moving up */
            while (p > 0 && row[best[p - 1]] > row[j]) {
                best[p] = best[p - 1];
                --p;
            }
            best[p] = j;
        }
    }
}

/* Tour length: sum of d over consecutive nodes, closing the cycle. */
ORC_API int64_t orc_tour_length(int32_t n, const int32_t *d, const int32_t *tour)
{
    int64_t len = 0;
    for (int32_t t = 0; t < n; ++t)
        len += d[(size_t)tour[t] * n + tour[(t + 1) % n]];
    return len;
}

/* Nearest-neighbour tour used for the initial trail limits (Sec. 2.1):
 * start at node 0, repeatedly move to the nearest unvisited node (ties -> lower id). */
ORC_API int64_t orc_nn_tour(int32_t n, const int32_t *d, int32_t *tour)
{
    uint8_t *vis = (uint8_t *)calloc((size_t)n, 1);
    int32_t cur = 0;
    tour[0] = 0;
    vis[0] = 1;
    for (int32_t t = 1; t < n; ++t) {
        int32_t best = -1;
        for (int32_t j = 0; j < n; ++j) {
            if (vis[j]) continue;
            if (best < 0 || d[(size_t)cur * n + j] < d[(size_t)cur * n + best]) best = j;
        }
        tour[t] = best;
        vis[best] = 1;
        cur = best;
    }
    free(vis);
    return orc_tour_length(n, d, tour);
}

/* Trail limits (reading R-lim, after Stuetzle and Hoos 2000, as Sec. 5 states):
 * tau_max = 1/(rho C); with p = p_best^(1/n) and avg = n/2,
 * tau_min = tau_max (1 - p) / ((avg - 1) p), capped at tau_max.
 * Computed in double and stored as float. */
ORC_API void orc_limits(int32_t n, double rho, double p_best, int64_t cost,
                        float *tmax_out, float *tmin_out)
{
    double tmax = 1.0 / (rho * (double)cost);
    double p = pow(p_best, 1.0 / (double)n);
    double avg = (double)n / 2.0;
    double tmin = tmax * (1.0 - p) / ((avg - 1.0) * p);
    if (tmin > tmax) tmin = tmax;
    *tmax_out = (float)tmax;
    *tmin_out = (float)tmin;
}

/* choice_info = tau^alpha * eta^beta, precomputed once per iteration (Sec. 2.1). */
ORC_API void orc_choice(int32_t n, const float *tau, const float *eb, double alpha, float *choice)
{
    for (size_t c = 0; c < (size_t)n * n; ++c) {
        double t = (double)tau[c];
        double ta = alpha == 1.0 ? t : pow(t, alpha);
        choice[c] = (float)(ta * (double)eb[c]);
    }
}

/* Evaporation (Sec. 2.1): tau <- max((1 - rho) tau, tau_min), every cell
 * (reading R-rho: `persist` is the float 1 - rho).  Reading R-bound: trails
 * stay inside [tau_min, tau_max] at all times (Sec. 2.1), so an evaporated
 * cell is also capped at tau_max; the cap only acts on the first iteration,
 * when the first global best is longer than the nearest-neighbour tour and
 * tau_max drops. */
ORC_API void orc_evaporate(int32_t n, float *tau, float persist, float tmin, float tmax)
{
    for (size_t c = 0; c < (size_t)n * n; ++c) {
        float e = (float)((double)tau[c] * (double)persist);
        e = e > tmin ? e : tmin;
        tau[c] = e < tmax ? e : tmax;
    }
}

/* Deposit (Sec. 2.1, Alg. 1): tau_ij <- min(tau_ij + Delta, tau_max) on every
 * edge (i,j) of the tour, in both directions (reading R-dep). */
ORC_API void orc_deposit(int32_t n, float *tau, const int32_t *tour, float delta, float tmax)
{
    for (int32_t t = 0; t < n; ++t) {
        int32_t a = tour[t], b = tour[(t + 1) % n];
        size_t ab = (size_t)a * n + b, ba = (size_t)b * n + a;
        float x = (float)((double)tau[ab] + (double)delta);
        tau[ab] = x < tmax ? x : tmax;
        x = (float)((double)tau[ba] + (double)delta);
        tau[ba] = x < tmax ? x : tmax;
    }
}

/* ------------------------------------------------------------------------ */
/* Node selection (Eq. (1); Sec. 4.2)                                       */
/* ------------------------------------------------------------------------ */

/* A-Res with a reservoir of one item (Alg. 3 with m = 1), in the logarithmic
 * form of Sec. 4.2.2: item i gets key log2(r_i) / w_i and the largest key wins;
 * the running best starts at -infinity.  Ties go to the lower id.
 * Returns the index into the arrays, or -1 when k == 0. */
ORC_API int32_t orc_wrs_pick(int32_t k, const int32_t *ids, const double *w, const double *r)
{
    int32_t best = -1;
    double bkey = -INFINITY;
    for (int32_t i = 0; i < k; ++i) {
        double key = log2(r[i]) / w[i];
        if (best < 0 || key > bkey || (key == bkey && ids[i] < ids[best])) {
            best = i;
            bkey = key;
        }
    }
    return best;
}

/* The roulette wheel (Sec. 4.2.1): node p of the k candidates is picked
 * with probability w_p / sum(w), by drawing theta = u * T (u uniform in
 * (0,1), T the sum of the weights) and walking the cumulative sums
 * C(p) = w_0 + ... + w_p until one exceeds theta.  The sums are taken in
 * double precision in position order; the winner is the first position
 * whose cumulative sum exceeds theta (a position of weight 0 can never be
 * that first one).  theta < T holds in double precision (u <= 1 - 2^-24), so
 * a winner always exists when some weight is positive; -1 when none is. */
ORC_API int32_t orc_rwm_pick(int32_t k, const double *w, double u)
{
    double total = 0.0;
    for (int32_t i = 0; i < k; ++i) total += w[i];
    if (!(total > 0.0)) return -1;
    const double theta = u * total;
    double acc = 0.0;
    int32_t last = -1;
    for (int32_t i = 0; i < k; ++i) {
        acc += w[i];
        if (w[i] > 0.0) last = i;
        if (theta < acc) return i;
    }
    return last;
}

ORC_API int64_t orc_two_opt(int32_t n, const int32_t *d, const int32_t *nn, int32_t k,
                            int32_t *tour);

/* ------------------------------------------------------------------------ */
/* The colony: Alg. 1                                                       */
/* ------------------------------------------------------------------------ */

typedef struct orc_colony {
    int32_t n, m, cl, deposit, fallback, ls;
    int32_t sel;       /* whole-row selection: 0 reservoir sampling, 1 roulette wheel */
    int32_t tabu;      /* whole-row tabu: 0 bitmask, 1 compact list (Sec. 4.1) */
    double alpha, beta, rho, p_best;
    float persist;
    uint64_t seed;
    int32_t *d;        /* n x n */
    float *eb;         /* n x n, eta^beta */
    int32_t *cand;     /* n x cl */
    float *tau;        /* n x n */
    float *choice;     /* n x n */
    float tmin, tmax;
    int32_t *tours;    /* m x n */
    int64_t *lens;     /* m */
    int64_t *fb;       /* m, fallback steps of the last construction */
    int32_t *best_tour;
    int64_t best_len;
    int32_t has_best;
    int32_t iter;      /* iterations completed */
    int64_t nn_len;
} orc_colony;

/* Build the colony: instance, heuristic weights, candidate lists, the
 * nearest-neighbour limits, tau <- tau_max and choice_info (Alg. 1 before the
 * main loop).  Exactly one of xy (n x 2) and dist (n x n) is non-NULL. */
ORC_API orc_colony *orc_colony_new(int32_t n, const int32_t *xy, const int32_t *dist, int32_t m,
                                   int32_t cl, double alpha, double beta, float rho,
                                   double p_best, uint64_t seed, int32_t deposit,
                                   int32_t fallback, int32_t ls)
{
    orc_colony *c = (orc_colony *)calloc(1, sizeof(orc_colony));
    size_t nn = (size_t)n * n;
    c->n = n; c->m = m; c->cl = cl; c->deposit = deposit; c->fallback = fallback; c->ls = ls;
    c->sel = 0; c->tabu = 0;
    c->alpha = alpha; c->beta = beta; c->rho = (double)rho; c->p_best = p_best;
    c->persist = (float)(1.0 - (double)rho);
    c->seed = seed;
    c->d = (int32_t *)malloc(sizeof(int32_t) * nn);
    if (xy) orc_distances(n, xy, c->d);
    else memcpy(c->d, dist, sizeof(int32_t) * nn);
    c->eb = (float *)malloc(sizeof(float) * nn);
    orc_eta_beta(n, c->d, beta, c->eb);
    c->cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (cl > 0 ? cl : 1));
    if (cl > 0) orc_candidates(n, c->d, cl, c->cand);
    int32_t *nn_tour = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    c->nn_len = orc_nn_tour(n, c->d, nn_tour);
    free(nn_tour);
    orc_limits(n, c->rho, p_best, c->nn_len, &c->tmax, &c->tmin);
    c->tau = (float *)malloc(sizeof(float) * nn);
    for (size_t i = 0; i < nn; ++i) c->tau[i] = c->tmax;
    c->choice = (float *)malloc(sizeof(float) * nn);
    orc_choice(n, c->tau, c->eb, alpha, c->choice);
    c->tours = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * n);
    c->lens = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    c->fb = (int64_t *)calloc((size_t)m, sizeof(int64_t));
    c->best_tour = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    c->best_len = 0;
    c->has_best = 0;
    c->iter = 0;
    return c;
}

ORC_API void orc_colony_free(orc_colony *c)
{
    if (!c) return;
    free(c->d); free(c->eb); free(c->cand); free(c->tau); free(c->choice);
    free(c->tours); free(c->lens); free(c->fb); free(c->best_tour);
    free(c);
}

/* Keys of every node that competes at step t of ant `ant` in iteration `it`,
 * standing at node i with the visited flags vis[] (Alg. 4, Eq. (1)).
 * keys[v] receives the reservoir key log2(r)/w of each competing node, or NaN
 * for nodes that do not compete.  For the greedy fallback (reading R-fb),
 * keys[v] receives choice_info[i][v] instead.
 * Returns 0 for a candidate-list draw, 1 for a full-row draw (no candidate
 * list, or fallback = 1 after the list was exhausted), 2 for the greedy fallback. */
ORC_API int32_t orc_step_keys(const orc_colony *c, int32_t it, int32_t ant, int32_t t, int32_t i,
                              const uint8_t *vis, double *keys)
{
    int32_t n = c->n;
    for (int32_t v = 0; v < n; ++v) keys[v] = NAN;
    if (c->cl > 0) {
        int any = 0;
        for (int32_t s = 0; s < c->cl; ++s) {
            int32_t v = c->cand[(size_t)i * c->cl + s];
            if (vis[v]) continue;
            double r = orc_uniform01(orc_word_cand(c->seed, it, ant, t, s));
            double w = (double)c->choice[(size_t)i * n + v];
            keys[v] = log2(r) / w;
            any = 1;
        }
        if (any) return 0;
        if (c->fallback == 0) {
            for (int32_t v = 0; v < n; ++v)
                if (!vis[v]) keys[v] = (double)c->choice[(size_t)i * n + v];
            return 2;
        }
    }
    for (int32_t v = 0; v < n; ++v) {
        if (vis[v]) continue;
        double r = orc_uniform01(orc_word_row(c->seed, it, ant, t, v));
        double w = (double)c->choice[(size_t)i * n + v];
        keys[v] = log2(r) / w;
    }
    return 1;
}

/* Largest key among the non-NaN entries, ties -> lower id. */
static int32_t argmax_keys(int32_t n, const double *keys)
{
    int32_t best = -1;
    for (int32_t v = 0; v < n; ++v) {
        if (isnan(keys[v])) continue;
        if (best < 0 || keys[v] > keys[best]) best = v;
    }
    return best;
}

/* Whole-row variants (cl = 0 only): selection 0 = reservoir sampling, 1 =
 * roulette wheel; tabu 0 = bitmask, 1 = compact list. */
ORC_API void orc_colony_set_variant(orc_colony *c, int32_t sel, int32_t tabu)
{
    c->sel = sel;
    c->tabu = tabu;
}

/* Remove node u from the compact list (Sec. 4.1): entries[0..L) are the
 * unvisited nodes; an unvisited node u < L sits at its own index, otherwise
 * entries[u] is the index it was moved to.  Its slot i_u is refilled by the
 * list's last node t = entries[L-1], whose new index is recorded at
 * entries[t]; when u is itself last, its slot takes the sentinel n. */
static void ct_remove(int32_t *entries, int32_t *L, int32_t n, int32_t u)
{
    const int32_t iu = u < *L ? u : entries[u];
    if (iu == *L - 1) {
        entries[iu] = n;
    } else {
        const int32_t t = entries[*L - 1];
        entries[iu] = t;
        entries[t] = iu;
    }
    --*L;
}

/* Step t of a whole-row variant from node cur over the npos selectable
 * positions, position p holding node order[p] (node order with visited nodes
 * flagged in vis for the bitmask; list order for the compact list).  Fills
 * val[p] with what the selection compares -- the weight choice_info (0 when
 * visited) for the roulette wheel, the key log2(r)/w (NaN when visited) for
 * reservoir sampling -- and returns the position picked:
 *   roulette wheel: orc_rwm_pick with u from orc_word_rwm (one draw per step);
 *   reservoir over the compact list: slot p's uniform from orc_word_slot,
 *     largest key, ties -> lower node id;
 *   reservoir over the bitmask: the plain whole-row keys of orc_step_keys. */
static int32_t variant_select(const orc_colony *c, int32_t it, int32_t ant, int32_t t, int32_t cur,
                              const int32_t *order, int32_t npos, const uint8_t *vis, double *val,
                              double *u_out)
{
    const float *row = c->choice + (size_t)cur * c->n;
    if (c->sel == 1) {
        for (int32_t p = 0; p < npos; ++p)
            val[p] = (vis && vis[order[p]]) ? 0.0 : (double)row[order[p]];
        const double u = orc_uniform01(orc_word_rwm(c->seed, it, ant, t));
        if (u_out) *u_out = u;
        return orc_rwm_pick(npos, val, u);
    }
    if (!c->tabu) {
        orc_step_keys(c, it, ant, t, cur, vis, val);
        return argmax_keys(c->n, val);
    }
    int32_t best = -1;
    for (int32_t p = 0; p < npos; ++p) {
        const double r = orc_uniform01(orc_word_slot(c->seed, it, ant, t, p));
        val[p] = log2(r) / (double)row[order[p]];
        if (best < 0 || val[p] > val[best] || (val[p] == val[best] && order[p] < order[best]))
            best = p;
    }
    return best;
}

/* A whole-row tour under the selected variant (cl = 0): the start node, then
 * n - 1 selections by variant_select, the compact list updated by ct_remove
 * or the bitmask by marking. */
static int64_t construct_row_variant(const orc_colony *c, int32_t it, int32_t ant, int32_t *tour)
{
    const int32_t n = c->n;
    uint8_t *vis = (uint8_t *)calloc((size_t)n, 1);
    int32_t *entries = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *val = (double *)malloc(sizeof(double) * (size_t)n);
    for (int32_t v = 0; v < n; ++v) entries[v] = v;
    int32_t L = n;
    int32_t cur = orc_start_node(c->seed, it, ant, n);
    tour[0] = cur;
    vis[cur] = 1;
    for (int32_t t = 1; t < n; ++t) {
        int32_t next;
        if (c->tabu) {
            ct_remove(entries, &L, n, cur);
            next = entries[variant_select(c, it, ant, t, cur, entries, L, NULL, val, NULL)];
        } else {
            next = variant_select(c, it, ant, t, cur, entries, n, vis, val, NULL);
        }
        tour[t] = next;
        vis[next] = 1;
        cur = next;
    }
    free(val);
    free(entries);
    free(vis);
    return orc_tour_length(n, c->d, tour);
}

/* Step t of ant `ant` in iteration `it` replayed on a given prefix of t nodes
 * (teacher forcing): rebuilds the tabu the prefix leaves (the compact list
 * by removing prefix[0..t) in order, or the visited set), writes the
 * selectable positions' nodes to order[], what the selection compares to
 * val[] and their count to *npos, the roulette wheel's draw to *u_out, and
 * returns the node the oracle picks.  Whole-row variants only. */
ORC_API int32_t orc_variant_step(const orc_colony *c, int32_t it, int32_t ant, const int32_t *prefix,
                                 int32_t t, int32_t *order, double *val, int32_t *npos, double *u_out)
{
    const int32_t n = c->n;
    const int32_t cur = prefix[t - 1];
    int32_t pick;
    *u_out = 0.0;
    if (c->tabu) {
        int32_t L = n;
        for (int32_t v = 0; v < n; ++v) order[v] = v;
        for (int32_t j = 0; j < t; ++j) ct_remove(order, &L, n, prefix[j]);
        *npos = L;
        pick = order[variant_select(c, it, ant, t, cur, order, L, NULL, val, u_out)];
    } else {
        uint8_t *vis = (uint8_t *)calloc((size_t)n, 1);
        for (int32_t j = 0; j < t; ++j) vis[prefix[j]] = 1;
        for (int32_t v = 0; v < n; ++v) order[v] = v;
        *npos = n;
        pick = variant_select(c, it, ant, t, cur, order, n, vis, val, u_out);
        free(vis);
    }
    return pick;
}

/* One ant's tour in iteration `it` (Alg. 1, inner loops): a random start, then
 * n-1 selections.  Returns the tour length; *fallbacks counts greedy or
 * full-row fallback steps taken after an exhausted candidate list. */
ORC_API int64_t orc_colony_construct(const orc_colony *c, int32_t it, int32_t ant, int32_t *tour,
                                     int64_t *fallbacks)
{
    if (c->cl == 0 && (c->sel != 0 || c->tabu != 0)) {
        if (fallbacks) *fallbacks = 0;
        return construct_row_variant(c, it, ant, tour);
    }
    int32_t n = c->n;
    uint8_t *vis = (uint8_t *)calloc((size_t)n, 1);
    double *keys = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t fb = 0;
    int32_t cur = orc_start_node(c->seed, it, ant, n);
    tour[0] = cur;
    vis[cur] = 1;
    for (int32_t t = 1; t < n; ++t) {
        int32_t mode = orc_step_keys(c, it, ant, t, cur, vis, keys);
        if (c->cl > 0 && mode != 0) ++fb;
        int32_t next = argmax_keys(n, keys);
        tour[t] = next;
        vis[next] = 1;
        cur = next;
    }
    free(keys);
    free(vis);
    if (fallbacks) *fallbacks = fb;
    return orc_tour_length(n, c->d, tour);
}

/* The part of Alg. 1's main loop after construction, given the iteration best
 * tour `ib_tour` of length `ib_len`: global best and trail limits (replaced
 * only by a strictly shorter tour), evaporation with the new limits, the
 * deposit on the iteration best (or the global best), choice_info, and the
 * iteration count. */
ORC_API void orc_colony_update(orc_colony *c, const int32_t *ib_tour, int64_t ib_len)
{
    int32_t n = c->n;
    if (!c->has_best || ib_len < c->best_len) {
        memcpy(c->best_tour, ib_tour, sizeof(int32_t) * (size_t)n);
        c->best_len = ib_len;
        c->has_best = 1;
        orc_limits(n, c->rho, c->p_best, c->best_len, &c->tmax, &c->tmin);
    }
    orc_evaporate(n, c->tau, c->persist, c->tmin, c->tmax);
    const int32_t *dep = c->deposit == 0 ? ib_tour : c->best_tour;
    int64_t dep_len = c->deposit == 0 ? ib_len : c->best_len;
    orc_deposit(n, c->tau, dep, (float)(1.0 / (double)dep_len), c->tmax);
    orc_choice(n, c->tau, c->eb, c->alpha, c->choice);
    c->iter += 1;
}

/* One iteration of Alg. 1's main loop.  Ants are independent given the
 * pheromone, so `threads` > 1 builds them concurrently (same results).
 * Local search (Sec. 5.7), with the candidate lists as neighbour lists:
 * ls = 1 improves the iteration best with 2-opt, ls = 2 every ant's tour. */
ORC_API void orc_colony_iterate(orc_colony *c, int32_t threads)
{
    int32_t n = c->n, m = c->m, it = c->iter;
    (void)threads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
    for (int32_t k = 0; k < m; ++k) {
        int32_t *t = c->tours + (size_t)k * n;
        c->lens[k] = orc_colony_construct(c, it, k, t, &c->fb[k]);
        if (c->ls == 2) {
            orc_two_opt(n, c->d, c->cand, c->cl, t);
            c->lens[k] = orc_tour_length(n, c->d, t);
        }
    }

    /* iteration best: shortest tour, ties -> lower ant index */
    int32_t ib = 0;
    for (int32_t k = 1; k < m; ++k)
        if (c->lens[k] < c->lens[ib]) ib = k;
    if (c->ls == 1) {
        int32_t *t = c->tours + (size_t)ib * n;
        orc_two_opt(n, c->d, c->cand, c->cl, t);
        c->lens[ib] = orc_tour_length(n, c->d, t);
    }
    orc_colony_update(c, c->tours + (size_t)ib * n, c->lens[ib]);
}

/* ---- accessors (copies out of the colony) ---- */
ORC_API int32_t orc_colony_iter(const orc_colony *c) { return c->iter; }
ORC_API int64_t orc_colony_nn_len(const orc_colony *c) { return c->nn_len; }
ORC_API int64_t orc_colony_best(const orc_colony *c, int32_t *tour)
{
    if (tour && c->has_best) memcpy(tour, c->best_tour, sizeof(int32_t) * (size_t)c->n);
    return c->has_best ? c->best_len : -1;
}
/* Replace the pheromone (n x n) and the trail limits, then choice_info, as
 * the set-up does: a state for tests to start the colony from. */
ORC_API void orc_colony_set_pheromone(orc_colony *c, const float *tau, float tmin, float tmax)
{
    memcpy(c->tau, tau, sizeof(float) * (size_t)c->n * c->n);
    c->tmin = tmin;
    c->tmax = tmax;
    orc_choice(c->n, c->tau, c->eb, c->alpha, c->choice);
}

ORC_API void orc_colony_limits(const orc_colony *c, float *tmin, float *tmax)
{
    *tmin = c->tmin;
    *tmax = c->tmax;
}
ORC_API void orc_colony_get(const orc_colony *c, int32_t *d, float *eb, int32_t *cand, float *tau,
                            float *choice)
{
    size_t nn = (size_t)c->n * c->n;
    if (d) memcpy(d, c->d, sizeof(int32_t) * nn);
    if (eb) memcpy(eb, c->eb, sizeof(float) * nn);
    if (cand && c->cl > 0) memcpy(cand, c->cand, sizeof(int32_t) * (size_t)c->n * c->cl);
    if (tau) memcpy(tau, c->tau, sizeof(float) * nn);
    if (choice) memcpy(choice, c->choice, sizeof(float) * nn);
}
ORC_API void orc_colony_tours(const orc_colony *c, int32_t *tours, int64_t *lens, int64_t *fb)
{
    if (tours) memcpy(tours, c->tours, sizeof(int32_t) * (size_t)c->m * c->n);
    if (lens) memcpy(lens, c->lens, sizeof(int64_t) * (size_t)c->m);
    if (fb) memcpy(fb, c->fb, sizeof(int64_t) * (size_t)c->m);
}

/* ------------------------------------------------------------------------ */
/* 2-opt local search (Sec. 5.7): Bentley's neighbour-list 2-opt with       */
/* don't-look bits, first improvement                                       */
/* ------------------------------------------------------------------------ */

/* Reverse the tour between positions a and b inclusive, going forward
 * (circularly) from a; keeps pos[] the inverse of tour[]. */
static void reverse_path(int32_t n, int32_t *tour, int32_t *pos, int32_t a, int32_t b)
{
    int32_t len = (b - a + n) % n + 1;
    for (int32_t s = 0; s < len / 2; ++s) {
        int32_t i = (a + s) % n, j = (b - s + n) % n;
        int32_t ci = tour[i], cj = tour[j];
        tour[i] = cj; pos[cj] = i;
        tour[j] = ci; pos[ci] = j;
    }
}

/* Apply the 2-opt move that removes edges (u1, v1) and (u2, v2), where v1
 * follows u1 and v2 follows u2 in tour order, and adds (u1, u2), (v1, v2):
 * reverse the path v1..u2, or -- when it is longer than half the tour --
 * the complementary path v2..u1, which gives the same cycle. */
static void apply_2opt(int32_t n, int32_t *tour, int32_t *pos, int32_t u1, int32_t v1, int32_t u2,
                       int32_t v2)
{
    int32_t a = pos[v1], b = pos[u2];
    int32_t len = (b - a + n) % n + 1;
    if (2 * len <= n) reverse_path(n, tour, pos, a, b);
    else reverse_path(n, tour, pos, pos[v2], pos[u1]);
}

/* The first improving 2-opt move at city c1 (Bentley 1992, as Sec. 5.7 says):
 * first with c1's successor s1, over c1's neighbours c2 in list order while
 * d(c1,c2) < d(c1,s1): gain d(c1,s1) + d(c2,s2) - d(c1,c2) - d(s1,s2), s2 the
 * successor of c2; then the same with predecessors.  Returns 1 and the move's
 * four cities (u1 -> v1 and u2 -> v2 are the removed edges in tour order), or
 * 0 when there is none. */
static int find_2opt(int32_t n, const int32_t *d, const int32_t *nn, int32_t k,
                     const int32_t *tour, const int32_t *pos, int32_t c1, int32_t mv[4])
{
    int32_t p = pos[c1];
    int32_t s1 = tour[(p + 1) % n], p1 = tour[(p - 1 + n) % n];
    int32_t radius = d[(size_t)c1 * n + s1];
    for (int32_t h = 0; h < k; ++h) {
        int32_t c2 = nn[(size_t)c1 * k + h];
        int32_t d12 = d[(size_t)c1 * n + c2];
        if (d12 >= radius) break;
        int32_t s2 = tour[(pos[c2] + 1) % n];
        int64_t gain = (int64_t)radius + d[(size_t)c2 * n + s2] - d12 - d[(size_t)s1 * n + s2];
        if (gain > 0) {
            mv[0] = c1; mv[1] = s1; mv[2] = c2; mv[3] = s2;
            return 1;
        }
    }
    radius = d[(size_t)p1 * n + c1];
    for (int32_t h = 0; h < k; ++h) {
        int32_t c2 = nn[(size_t)c1 * k + h];
        int32_t d12 = d[(size_t)c1 * n + c2];
        if (d12 >= radius) break;
        int32_t p2 = tour[(pos[c2] - 1 + n) % n];
        int64_t gain = (int64_t)radius + d[(size_t)p2 * n + c2] - d12 - d[(size_t)p1 * n + p2];
        if (gain > 0) {
            /* removed edges p1 -> c1 and p2 -> c2 */
            mv[0] = p2; mv[1] = c2; mv[2] = p1; mv[3] = c1;
            return 1;
        }
    }
    return 0;
}

/* 2-opt to a local optimum of the neighbour-list neighbourhood.  A run starts
 * with every don't-look bit clear and makes passes over the cities in index
 * order, skipping cities whose bit is set; a city without a move gets its bit
 * set, a move clears the bits of its four cities; the run ends after a pass
 * without a move.  Don't-look bits can hide a move that appeared after a
 * city's bit was set, so runs repeat until a whole run makes no move.
 * Returns the number of moves; the tour is improved in place. */
ORC_API int64_t orc_two_opt(int32_t n, const int32_t *d, const int32_t *nn, int32_t k,
                            int32_t *tour)
{
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t *dlb = (uint8_t *)malloc((size_t)n);
    for (int32_t i = 0; i < n; ++i) pos[tour[i]] = i;
    int64_t moves = 0;
    for (;;) {
        memset(dlb, 0, (size_t)n);
        int64_t run_moves = 0;
        int improved = 1;
        while (improved) {
            improved = 0;
            for (int32_t c1 = 0; c1 < n; ++c1) {
                if (dlb[c1]) continue;
                int32_t mv[4];
                if (find_2opt(n, d, nn, k, tour, pos, c1, mv)) {
                    apply_2opt(n, tour, pos, mv[0], mv[1], mv[2], mv[3]);
                    for (int q = 0; q < 4; ++q) dlb[mv[q]] = 0;
                    improved = 1;
                    ++run_moves;
                } else {
                    dlb[c1] = 1;
                }
            }
        }
        moves += run_moves;
        if (run_moves == 0) break;
    }
    free(pos);
    free(dlb);
    return moves;
}

/* ------------------------------------------------------------------------ */
/* Exact optimum by enumeration (n <= 11), for pinning tour quality         */
/* ------------------------------------------------------------------------ */

/* Every tour that starts at node 0: (n-1)! permutations of the others, in
 * lexicographic order.  Returns the shortest length and one shortest tour. */
ORC_API int64_t orc_brute_force(int32_t n, const int32_t *d, int32_t *best_tour)
{
    int32_t perm[16];
    int64_t best = -1;
    if (n < 2 || n > 12) return -1;
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (;;) {
        int64_t len = orc_tour_length(n, d, perm);
        if (best < 0 || len < best) {
            best = len;
            memcpy(best_tour, perm, sizeof(int32_t) * (size_t)n);
        }
        /* next permutation of perm[1..n-1] */
        int32_t i = n - 2;
        while (i >= 1 && perm[i] > perm[i + 1]) --i;
        if (i < 1) break;
        int32_t j = n - 1;
        while (perm[j] < perm[i]) --j;
        int32_t tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
        for (int32_t a = i + 1, b = n - 1; a < b; ++a, --b) {
            tmp = perm[a]; perm[a] = perm[b]; perm[b] = tmp;
        }
    }
    return best;
}
