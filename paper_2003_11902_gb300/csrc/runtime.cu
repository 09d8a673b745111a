// Host runtime behind the C ABI declared in include/mmas.h.
//
// A handle owns every device buffer of one colony, the stream it enqueues on
// and a CUDA graph holding one iteration of Alg. 1 (construction -> best and
// limits -> fused pheromone pass).  The iteration index, limits and best
// lengths live in device memory, so graph replays need no host round trip.
//
// Device layout (ld = n rounded up to 32; every n x n matrix row starts on a
// 128-byte boundary):
//   dist  int32 [n][ld]    eb   float [n][ld]    tau  float [n][ld]
//   wmat  float [n][ld]    choice_info (cl > 0) or 1/choice_info (cl = 0)
//   cand32 int32 [n][cl]   cand16 uint16 [n][cl]   cwinv float [n][cl]
//   tours int32 [m][ld]    lens int32 [m]   gb_tour int32 [n]   nbr int2 [n]
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <climits>
#include <new>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace mmas;

namespace {

thread_local std::string tl_error;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Armed by mmas_debug_fail_allocation: device allocations to let through
// before one fails (-1: none fails).
std::atomic<int> g_fail_after{-1};

mmas_status fail(mmas_handle *h, mmas_status st, const std::string &msg)
{
    if (h)
        h->err = msg;
    else
        tl_error = msg;
    return st;
}

#define CK(h, call)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail((h), e_ == cudaErrorMemoryAllocation ? MMAS_ENOMEM : MMAS_ECUDA,    \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

size_t pad16(size_t b) { return (b + 15) & ~size_t(15); }

void free_all(mmas_handle *h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (cudaEvent_t &e : h->ev)
        if (e) cudaEventDestroy(e);
    void *bufs[] = {h->xy,      h->dist,   h->eb,      h->tau,     h->wmat, h->cwinv,
                    h->cand32,  h->cand16, h->tours,   h->lens,    h->gb_tour, h->nn_tour,
                    h->nbr,     h->sc,     h->maxd,    h->ext_tour, h->ext_len, h->ext_bad, h->nnd,
                    h->xl32,    h->xlw,    h->xlb,     h->xxw,     h->xxn,  h->xhot,
                    h->xf16,    h->xfb,    h->far,     h->ebt};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (h->h_sc) cudaFreeHost(h->h_sc);
    if (h->h_tour) cudaFreeHost(h->h_tour);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// Allocate and zero a device buffer; the zeroing is ordered on `stream`, the
// stream every later kernel of the handle runs on (a plain cudaMemset would run
// on the legacy stream, unordered with a non-blocking one).
template <typename T>
cudaError_t dalloc(T **p, size_t bytes, cudaStream_t stream)
{
    cudaError_t e = device_malloc(reinterpret_cast<void **>(p), bytes ? bytes : 16);
    if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes ? bytes : 16, stream);
    return e;
}

// Read back the scalar block (with `tour` set, also the best tour into the
// pinned staging buffer, in the same synchronisation) and turn device-raised
// error bits into a status.
mmas_status sync_and_check(mmas_handle *h, bool tour = false)
{
    CK(h, cudaMemcpyAsync(h->h_sc, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
    if (tour)
        CK(h, cudaMemcpyAsync(h->h_tour, h->gb_tour, (size_t)h->n * 4, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const uint32_t e = h->h_sc->err;
    if (e) {
        const uint32_t zero = 0;
        cudaMemcpy(&h->sc->err, &zero, sizeof(zero), cudaMemcpyHostToDevice);
        if (e & ERR_STAGE_TIMEOUT)
            return fail(h, MMAS_ETIMEOUT, "a shared-memory staging wait on the device timed out");
        if (e & ERR_LS_CAP)
            return fail(h, MMAS_ESTATE, "a 2-opt search exceeded its move cap and stopped early");
        if (e & ERR_BAD_TOUR)
            return fail(h, MMAS_ESTATE, "a device-side tour given to mmas_update_device was not a permutation "
                                        "of 0..n-1 (or its length not positive); that update was skipped");
        return fail(h, MMAS_ESTATE, "the device found no unvisited node during a selection");
    }
    return MMAS_OK;
}

mmas_status validate(const mmas_instance *inst, const mmas_params *p)
{
    if (!inst || !p) return fail(nullptr, MMAS_EINVAL, "instance and params must be non-NULL");
    const int n = inst->n;
    if (n < 3 || n > 65535) return fail(nullptr, MMAS_EINVAL, "n must be in [3, 65535]");
    if ((inst->xy == nullptr) == (inst->dist == nullptr))
        return fail(nullptr, MMAS_EINVAL, "exactly one of xy and dist must be given");
    if (p->m < 1 || p->m > (1 << 20)) return fail(nullptr, MMAS_EINVAL, "m must be in [1, 2^20]");
    if (!(p->alpha >= 0.0f) || !std::isfinite(p->alpha))
        return fail(nullptr, MMAS_EINVAL, "alpha must be finite and >= 0");
    if (!(p->beta >= 0.0f) || !std::isfinite(p->beta))
        return fail(nullptr, MMAS_EINVAL, "beta must be finite and >= 0");
    if (!(p->rho > 0.0f && p->rho < 1.0f)) return fail(nullptr, MMAS_EINVAL, "rho must be in (0, 1)");
    if (!(p->p_best > 0.0f && p->p_best < 1.0f))
        return fail(nullptr, MMAS_EINVAL, "p_best must be in (0, 1)");
    if (p->cl < 0 || p->cl > 64 || p->cl >= n)
        return fail(nullptr, MMAS_EINVAL, "cl must be in [0, min(64, n - 1)]");
    if (p->ls != 0 && p->cl > 32)
        return fail(nullptr, MMAS_EINVAL, "local search uses the candidate lists as neighbour lists: cl <= 32");
    if (p->deposit != 0 && p->deposit != 1) return fail(nullptr, MMAS_EINVAL, "deposit must be 0 or 1");
    if (p->fallback != 0 && p->fallback != 1)
        return fail(nullptr, MMAS_EINVAL, "fallback must be 0 or 1");
    if (p->ant_offset < 0 || (long long)p->ant_offset + p->m > INT_MAX)
        return fail(nullptr, MMAS_EINVAL, "ant_offset must be >= 0 and ant_offset + m < 2^31");
    if (p->ls < 0 || p->ls > 2) return fail(nullptr, MMAS_EINVAL, "ls must be 0, 1 or 2");
    if (p->selection < 0 || p->selection > 1) return fail(nullptr, MMAS_EINVAL, "selection must be 0 or 1");
    if (p->tabu < 0 || p->tabu > 1) return fail(nullptr, MMAS_EINVAL, "tabu must be 0 or 1");
    if ((p->selection || p->tabu) && p->cl != 0)
        return fail(nullptr, MMAS_EINVAL, "selection and tabu variants are whole-row (cl = 0) variants");
    if (p->ls > 0 && p->cl < 1)
        return fail(nullptr, MMAS_EINVAL, "ls needs candidate lists (cl >= 1) as neighbour lists");
    if (inst->xy) {
        for (int i = 0; i < 2 * n; ++i) {
            const long long c = inst->xy[i];
            if (c <= -(1ll << 30) || c >= (1ll << 30))
                return fail(nullptr, MMAS_EINVAL, "coordinates must satisfy |x|, |y| < 2^30");
        }
    } else {
        const int32_t *d = inst->dist;
        for (int i = 0; i < n; ++i) {
            if (d[(size_t)i * n + i] != 0) return fail(nullptr, MMAS_EINVAL, "dist must have a zero diagonal");
            for (int j = 0; j < n; ++j) {
                const int32_t v = d[(size_t)i * n + j];
                if (v < 0) return fail(nullptr, MMAS_EINVAL, "dist must be non-negative");
                if (v != d[(size_t)j * n + i]) return fail(nullptr, MMAS_EINVAL, "dist must be symmetric");
            }
        }
    }
    return MMAS_OK;
}

// Record one iteration (construct -> best -> update) as a CUDA graph, with
// event-record nodes at the phase boundaries when phase timing is on.
mmas_status capture_iteration(mmas_handle *h)
{
    cudaStream_t cs;
    CK(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess && h->timing) e = cudaEventRecordWithFlags(h->ev[0], cs, cudaEventRecordExternal);
    if (e == cudaSuccess) e = launch_construct(h->cargs, h->cplan, cs);
    if (e == cudaSuccess && h->timing) e = cudaEventRecordWithFlags(h->ev[1], cs, cudaEventRecordExternal);
    if (h->p.ls == 1) {
        // lengths, 2-opt of the iteration best, then best / limits
        ScoreArgs sa = h->sargs;
        sa.best = 0;
        if (e == cudaSuccess) e = launch_score(sa, h->num_sms, cs);
        if (e == cudaSuccess) e = launch_two_opt(h->targs, true, h->num_sms, h->smem_optin, cs);
        if (e == cudaSuccess) e = launch_best(h->bargs, cs);
    } else {
        if (h->p.ls == 2 && e == cudaSuccess) e = launch_two_opt(h->targs, false, h->num_sms, h->smem_optin, cs);
        if (e == cudaSuccess) e = launch_score(h->sargs, h->num_sms, cs);
    }
    if (e == cudaSuccess) e = launch_update(h->uargs, h->num_sms, cs);
    if (e == cudaSuccess && h->timing) e = cudaEventRecordWithFlags(h->ev[2], cs, cudaEventRecordExternal);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(h, MMAS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(h, MMAS_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->graph = g;
    h->gexec = ge;
    return MMAS_OK;
}

mmas_status create_impl(mmas_handle *h, const mmas_instance *inst)
{
    const int n = h->n, m = h->m, cl = h->cl, ld = h->ld;
    cudaDeviceProp prop;
    CK(h, cudaGetDeviceProperties(&prop, h->device));
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(h, MMAS_ECUDA, std::string("libmmas is built for sm_103a; device ") + prop.name +
                                       " is sm_" + std::to_string(prop.major) + std::to_string(prop.minor));
    h->num_sms = prop.multiProcessorCount;
    h->smem_optin = prop.sharedMemPerBlockOptin;
    if (h->p.stream) {
        h->stream = static_cast<cudaStream_t>(h->p.stream);
    } else {
        CK(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }

    const size_t nn = (size_t)n * ld;
    size_t need = nn * 4 * 4 + (size_t)m * ld * 4;
    size_t free_b = 0, total_b = 0;
    CK(h, cudaMemGetInfo(&free_b, &total_b));
    if (need + (64u << 20) > free_b)
        return fail(h, MMAS_ENOMEM, "not enough device memory for the n x n matrices and tours");

    const size_t cw_bytes = pad16((size_t)n * (cl ? cl : 1) * sizeof(float));
    const size_t cc_bytes = pad16((size_t)n * (cl ? cl : 1) * sizeof(uint16_t));
    CK(h, dalloc(&h->dist, nn * sizeof(int32_t), h->stream));
    CK(h, dalloc(&h->eb, nn * sizeof(float), h->stream));
    CK(h, dalloc(&h->tau, nn * sizeof(float), h->stream));
    CK(h, dalloc(&h->wmat, nn * sizeof(float), h->stream));
    CK(h, dalloc(&h->cand32, (size_t)n * (cl ? cl : 1) * sizeof(int32_t), h->stream));
    CK(h, dalloc(&h->cand16, cc_bytes, h->stream));
    CK(h, dalloc(&h->cwinv, cw_bytes, h->stream));
    CK(h, dalloc(&h->tours, (size_t)m * ld * sizeof(int32_t), h->stream));
    CK(h, dalloc(&h->lens, (size_t)m * sizeof(int32_t), h->stream));
    CK(h, dalloc(&h->gb_tour, (size_t)n * sizeof(int32_t), h->stream));
    CK(h, dalloc(&h->nn_tour, (size_t)n * sizeof(int32_t), h->stream));
    CK(h, dalloc(&h->nbr, (size_t)n * sizeof(int2), h->stream));
    CK(h, dalloc(&h->sc, sizeof(Scalars), h->stream));
    CK(h, dalloc(&h->maxd, sizeof(int), h->stream));
    CK(h, dalloc(&h->ext_tour, (size_t)n * sizeof(int32_t), h->stream));
    CK(h, dalloc(&h->ext_len, sizeof(int32_t), h->stream));
    CK(h, dalloc(&h->ext_bad, sizeof(uint32_t), h->stream));
    CK(h, cudaMallocHost(reinterpret_cast<void **>(&h->h_sc), sizeof(Scalars)));
    CK(h, cudaMallocHost(reinterpret_cast<void **>(&h->h_tour), (size_t)n * sizeof(int32_t)));
    std::memset(h->h_sc, 0, sizeof(Scalars));

    // instance -> device, distances, overflow check
    cudaStream_t s = h->stream;
    if (inst->xy) {
        CK(h, dalloc(&h->xy, (size_t)n * sizeof(int2), h->stream));
        CK(h, cudaMemcpyAsync(h->xy, inst->xy, (size_t)n * sizeof(int2), cudaMemcpyHostToDevice, s));
        CK(h, launch_distances(h->xy, n, ld, h->dist, h->maxd, s));
    } else {
        CK(h, cudaMemcpy2DAsync(h->dist, (size_t)ld * 4, inst->dist, (size_t)n * 4, (size_t)n * 4, n,
                                cudaMemcpyHostToDevice, s));
        CK(h, launch_max_dist(h->dist, n, ld, h->maxd, s));
    }
    int maxd = 0;
    CK(h, cudaMemcpyAsync(&maxd, h->maxd, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    if ((long long)n * (long long)maxd >= (1ll << 31))
        return fail(h, MMAS_EOVERFLOW, "n * max distance must be < 2^31 (32-bit tour lengths)");

    // scalars: no global best yet
    Scalars init{};
    init.gb_len = INT_MAX;
    init.ib_len = -1;
    init.ib_ant = -1;
    *h->h_sc = init;
    CK(h, cudaMemcpyAsync(h->sc, h->h_sc, sizeof(Scalars), cudaMemcpyHostToDevice, s));

    h->maxd_val = maxd;
    if (maxd <= ETA_TABLE_MAX) CK(h, dalloc(&h->ebt, ((size_t)maxd + 1) * sizeof(float), h->stream));
    CK(h, launch_eta_beta(h->dist, n, ld, (double)h->p.beta, h->eb, h->ebt, h->maxd_val, s));
    CK(h, launch_candidates(h->dist, n, ld, cl, h->cand32, h->cand16, s));
    // greedy fallback (fallback 0): a reach list of the min(REACH_MAX, n - 1)
    // nearest nodes per row, refreshed with choice_info, usually decides it
    // without a row scan
    if (cl > 0 && h->p.fallback == 0 && n - 1 > cl) {
        h->xe = n - 1 < REACH_MAX ? n - 1 : REACH_MAX;
        CK(h, dalloc(&h->xl32, (size_t)n * h->xe * sizeof(int32_t), h->stream));
        CK(h, dalloc(&h->xlw, (size_t)n * h->xe * sizeof(uint2), h->stream));
        CK(h, dalloc(&h->xlb, (size_t)n * sizeof(float), h->stream));
        CK(h, dalloc(&h->xxw, (size_t)n * REACH_EXTRA * sizeof(uint2), h->stream));
        CK(h, dalloc(&h->xxn, (size_t)n * sizeof(int32_t), h->stream));
        CK(h, dalloc(&h->xhot, (size_t)n * sizeof(int32_t), h->stream));
        CK(h, launch_candidates(h->dist, n, ld, h->xe, h->xl32, nullptr, s));
        // large rows: the far list (the nearest REACH_FAR nodes, 16-bit ids) and
        // its bound decide most fallbacks the reach list cannot
        if (n >= REACH_FAR_MIN_N) {
            h->fp = REACH_FAR;
            h->fe = REACH_FAR - REACH_MAX;
            CK(h, dalloc(&h->xf16, (size_t)n * h->fp * sizeof(uint16_t), h->stream));
            CK(h, dalloc(&h->xfb, (size_t)n * sizeof(float), h->stream));
            CK(h, launch_candidates(h->dist, n, ld, h->fp, nullptr, h->xf16, s));
            CK(h, dalloc(&h->far, sizeof(FarList), h->stream));
            const FarList fl{h->xf16, h->xfb, h->fp, 0};
            CK(h, cudaMemcpyAsync(h->far, &fl, sizeof(fl), cudaMemcpyHostToDevice, s));
            CK(h, cudaStreamSynchronize(s));  // fl is on the host stack
        }
    }
    // the nearest-neighbour tour reads the longest sorted list there is
    if (h->xf16)
        CK(h, launch_nn_tour(h->dist, n, ld, h->nn_tour, h->sc, h->xf16, true, h->fp, h->fp, s));
    else if (h->xl32)
        CK(h, launch_nn_tour(h->dist, n, ld, h->nn_tour, h->sc, h->xl32, false, h->xe, h->xe, s));
    else
        CK(h, launch_nn_tour(h->dist, n, ld, h->nn_tour, h->sc, cl > 0 ? h->cand32 : nullptr, false, cl, cl, s));
    CK(h, launch_init_colony(n, ld, (double)h->p.rho, h->p_root, h->tau, h->sc, s));

    // launch arguments of one iteration
    ConstructArgs &ca = h->cargs;
    ca.n = n; ca.m = m; ca.cl = cl; ca.ld = ld; ca.fallback = h->p.fallback;
    ca.ant_offset = h->p.ant_offset;
    ca.sel = h->p.selection;
    ca.ct = h->p.tabu;
    ca.key0 = (uint32_t)(h->p.seed & 0xFFFFFFFFull);
    ca.key1 = (uint32_t)(h->p.seed >> 32);
    for (int r = 0; r < 10; ++r) {
        ca.rk0[r] = ca.key0 + (uint32_t)r * 0x9E3779B9u;
        ca.rk1[r] = ca.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    ca.iter = &h->sc->iter;
    ca.cand16 = h->cand16; ca.cwinv = h->cwinv; ca.wmat = h->wmat;
    ca.tours = h->tours; ca.sc = h->sc;
    ca.xe = h->xe; ca.xlw = h->xlw; ca.xlb = h->xlb; ca.xxw = h->xxw; ca.xxn = h->xxn;
    ca.far = h->far;
    ca.stage_w_bytes = (uint32_t)cw_bytes;
    ca.stage_c_bytes = (uint32_t)cc_bytes;
    if (cl == 0) { ca.stage_w_bytes = 0; ca.stage_c_bytes = 0; }
    CK(h, plan_construct(ca, h->num_sms, h->smem_optin, &h->cplan));

    BestArgs &ba = h->bargs;
    ba.n = n; ba.m = m; ba.ld = ld; ba.deposit = h->p.deposit; ba.advance = 1;
    ba.rho = (double)h->p.rho; ba.p_root = h->p_root;
    ba.lens = h->lens; ba.tours = h->tours; ba.gb_tour = h->gb_tour; ba.nbr = h->nbr; ba.sc = h->sc;

    ScoreArgs &sa = h->sargs;
    sa.n = n; sa.m = m; sa.ld = ld; sa.best = 1;
    sa.tours = h->tours; sa.xy = h->xy; sa.dist = h->dist; sa.lens = h->lens; sa.b = ba;

    TwoOptArgs &ta = h->targs;
    ta.n = n; ta.m = m; ta.ld = ld; ta.k = cl;
    ta.nn = h->cand32; ta.nn16 = h->cand16; ta.xy = h->xy; ta.dist = h->dist; ta.tours = h->tours; ta.lens = h->lens;
    ta.err = &h->sc->err;
    if (h->p.ls > 0 && !two_opt_fits(n, cl, false, (size_t)h->smem_optin))
        return fail(h, MMAS_EINVAL, "ls needs about 12.1n bytes of shared memory per CTA: n is too large");
    if (h->p.ls > 0) {
        CK(h, dalloc(&h->nnd, (size_t)n * cl * sizeof(int32_t), h->stream));
        CK(h, launch_neighbour_dist(ta, h->nnd, s));
        ta.nnd = h->nnd;
    }

    UpdateArgs &ua = h->uargs;
    ua.n = n; ua.ld = ld; ua.cl = cl; ua.fullrow = cl == 0; ua.evaporate = 1;
    ua.recip = cl == 0 && h->p.selection == 0;
    ua.persist = (float)(1.0 - (double)h->p.rho);
    ua.alpha = h->p.alpha;
    ua.eb = h->eb; ua.tau = h->tau; ua.wmat = h->wmat; ua.cand32 = h->cand32; ua.cwinv = h->cwinv;
    ua.nbr = h->nbr; ua.sc = h->sc;
    ua.xe = h->xe; ua.xl32 = h->xl32; ua.xlw = h->xlw; ua.xlb = h->xlb; ua.xxw = h->xxw; ua.xxn = h->xxn;
    ua.xhot = h->xhot;
    ua.fe = h->fe; ua.fp = h->fp; ua.xf16 = h->xf16; ua.xfb = h->xfb;

    // choice_info of the initial pheromone
    UpdateArgs refresh = ua;
    refresh.evaporate = 0;
    refresh.nbr = nullptr;
    CK(h, launch_update(refresh, h->num_sms, s));

    mmas_status st = capture_iteration(h);
    if (st != MMAS_OK) return st;
    return sync_and_check(h);
}

mmas_status check_handle(mmas_handle *h)
{
    if (!h) return fail(nullptr, MMAS_EINVAL, "handle is NULL");
    return MMAS_OK;
}

}  // namespace

void mmas::set_thread_error(const std::string &msg) { tl_error = msg; }

cudaError_t mmas::device_malloc(void **p, size_t bytes)
{
    int v = g_fail_after.load();
    while (v >= 0) {
        if (g_fail_after.compare_exchange_weak(v, v == 0 ? -1 : v - 1)) {
            if (v == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

mmas_status mmas::validate_colony(const mmas_instance *inst, const mmas_params *params)
{
    mmas_params p = *params;
    if (p.m == 0) p.m = inst->n;
    return validate(inst, &p);
}

extern "C" {

void mmas_debug_fail_allocation(int32_t after) { g_fail_after.store(after < 0 ? -1 : after); }

mmas_status mmas_debug_two_opt_move_cap(int32_t device, int64_t cap)
{
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(nullptr, MMAS_EINVAL, "device ordinal out of range");
    DeviceGuard g(device);
    const cudaError_t e = set_two_opt_move_cap(cap);
    if (e != cudaSuccess) return fail(nullptr, MMAS_ECUDA, std::string("set_two_opt_move_cap: ") + cudaGetErrorString(e));
    return MMAS_OK;
}

mmas_status mmas_debug_expire_stage_waits(int32_t device, int32_t on)
{
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(nullptr, MMAS_EINVAL, "device ordinal out of range");
    DeviceGuard g(device);
    const cudaError_t e = set_stage_wait_expiry(on != 0);
    if (e != cudaSuccess) return fail(nullptr, MMAS_ECUDA, std::string("set_stage_wait_expiry: ") + cudaGetErrorString(e));
    return MMAS_OK;
}

void mmas_default_params(mmas_params *p)
{
    if (!p) return;
    p->m = 0;
    p->alpha = 1.0f;
    p->beta = 2.0f;
    p->rho = 0.02f;
    p->p_best = 0.01f;
    p->cl = 32;
    p->seed = 1;
    p->deposit = 0;
    p->fallback = 0;
    p->device = 0;
    p->ant_offset = 0;
    p->ls = 0;
    p->selection = 0;
    p->tabu = 0;
    p->stream = nullptr;
}

mmas_status mmas_create(const mmas_instance *inst, const mmas_params *p_in, mmas_handle **out)
{
    if (!out) return fail(nullptr, MMAS_EINVAL, "out must be non-NULL");
    *out = nullptr;
    tl_error.clear();
    if (!inst || !p_in) return fail(nullptr, MMAS_EINVAL, "instance and params must be non-NULL");
    mmas_params p = *p_in;
    if (p.m == 0) p.m = inst->n;
    mmas_status st = validate(inst, &p);
    if (st != MMAS_OK) return st;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(nullptr, MMAS_ECUDA, "no CUDA device is available");
    if (p.device < 0 || p.device >= ndev) return fail(nullptr, MMAS_EINVAL, "device ordinal out of range");

    mmas_handle *h = new (std::nothrow) mmas_handle();
    if (!h) return fail(nullptr, MMAS_ENOMEM, "host allocation failed");
    h->device = p.device;
    h->p = p;
    h->n = inst->n;
    h->m = p.m;
    h->cl = p.cl;
    h->ld = (inst->n + 31) & ~31;
    h->p_root = std::pow((double)p.p_best, 1.0 / (double)inst->n);
    DeviceGuard g(h->device);
    st = create_impl(h, inst);
    if (st != MMAS_OK) {
        tl_error = h->err;
        if (h->stream) cudaStreamSynchronize(h->stream);
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return MMAS_OK;
}

mmas_status mmas_iterate(mmas_handle *h, int32_t k)
{
    if (check_handle(h)) return MMAS_EINVAL;
    if (k < 0) return fail(h, MMAS_EINVAL, "k must be >= 0");
    DeviceGuard g(h->device);
    for (int32_t i = 0; i < k; ++i) CK(h, cudaGraphLaunch(h->gexec, h->stream));
    if (k > 0 && h->timing) h->timed_run = true;
    return MMAS_OK;
}

mmas_status mmas_best_tour(mmas_handle *h, int32_t *tour_out, int32_t *len_out)
{
    if (check_handle(h)) return MMAS_EINVAL;
    DeviceGuard g(h->device);
    mmas_status st = sync_and_check(h, tour_out != nullptr);
    if (st != MMAS_OK) return st;
    if (h->h_sc->gb_len == INT_MAX) return fail(h, MMAS_ESTATE, "no iteration has completed yet");
    if (tour_out) std::memcpy(tour_out, h->h_tour, (size_t)h->n * 4);
    if (len_out) *len_out = h->h_sc->gb_len;
    return MMAS_OK;
}

void mmas_destroy(mmas_handle *h)
{
    if (!h) return;
    DeviceGuard g(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

const char *mmas_last_error(const mmas_handle *h)
{
    return h ? h->err.c_str() : tl_error.c_str();
}

mmas_status mmas_construct(mmas_handle *h)
{
    if (check_handle(h)) return MMAS_EINVAL;
    DeviceGuard g(h->device);
    CK(h, launch_construct(h->cargs, h->cplan, h->stream));
    ScoreArgs sa = h->sargs;
    sa.best = 0;
    CK(h, launch_score(sa, h->num_sms, h->stream));
    return MMAS_OK;
}

mmas_status mmas_two_opt_tour(mmas_handle *h, int32_t *tour, int32_t *len_out)
{
    if (check_handle(h)) return MMAS_EINVAL;
    if (!tour) return fail(h, MMAS_EINVAL, "tour must be non-NULL");
    if (h->cl < 1 || h->cl > 32) return fail(h, MMAS_EINVAL, "2-opt uses the candidate lists: 1 <= cl <= 32");
    if (!two_opt_fits(h->n, h->cl, false, (size_t)h->smem_optin))
        return fail(h, MMAS_EINVAL, "2-opt needs about 12.1n bytes of shared memory per CTA: n is too large");
    std::vector<char> seen((size_t)h->n, 0);
    for (int i = 0; i < h->n; ++i) {
        const int v = tour[i];
        if (v < 0 || v >= h->n || seen[v]) return fail(h, MMAS_EINVAL, "tour must be a permutation of 0..n-1");
        seen[v] = 1;
    }
    DeviceGuard g(h->device);
    if (!h->nnd) {  // neighbour distances, once, as a colony with local search has them
        CK(h, dalloc(&h->nnd, (size_t)h->n * h->cl * sizeof(int32_t), h->stream));
        CK(h, launch_neighbour_dist(h->targs, h->nnd, h->stream));
        h->targs.nnd = h->nnd;
    }
    CK(h, cudaMemcpyAsync(h->ext_tour, tour, (size_t)h->n * 4, cudaMemcpyHostToDevice, h->stream));
    TwoOptArgs ta = h->targs;
    ta.m = 1;
    ta.tours = h->ext_tour;
    ta.lens = h->ext_len;
    CK(h, launch_two_opt(ta, false, h->num_sms, (int)h->smem_optin, h->stream));
    int32_t len = 0;
    CK(h, cudaMemcpyAsync(tour, h->ext_tour, (size_t)h->n * 4, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(&len, h->ext_len, sizeof(len), cudaMemcpyDeviceToHost, h->stream));
    mmas_status st = sync_and_check(h);
    if (st != MMAS_OK) return st;
    if (len_out) *len_out = len;
    return MMAS_OK;
}

mmas_status mmas_update(mmas_handle *h, const int32_t *tour, int32_t len)
{
    if (check_handle(h)) return MMAS_EINVAL;
    if (!tour || len <= 0) return fail(h, MMAS_EINVAL, "tour must be non-NULL and len > 0");
    std::vector<char> seen((size_t)h->n, 0);
    for (int i = 0; i < h->n; ++i) {
        const int v = tour[i];
        if (v < 0 || v >= h->n || seen[v]) return fail(h, MMAS_EINVAL, "tour must be a permutation of 0..n-1");
        seen[v] = 1;
    }
    DeviceGuard g(h->device);
    CK(h, cudaMemcpyAsync(h->ext_tour, tour, (size_t)h->n * 4, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->ext_len, &len, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    BestArgs b = h->bargs;
    b.m = 1;
    b.lens = h->ext_len;
    b.tours = h->ext_tour;
    b.advance = 0;
    CK(h, launch_best(b, h->stream));
    CK(h, launch_update(h->uargs, h->num_sms, h->stream));
    return MMAS_OK;
}

mmas_status mmas_get_tours(mmas_handle *h, int32_t *tours, int32_t *lens)
{
    if (check_handle(h)) return MMAS_EINVAL;
    DeviceGuard g(h->device);
    mmas_status st = sync_and_check(h);
    if (st != MMAS_OK) return st;
    if (tours)
        CK(h, cudaMemcpy2D(tours, (size_t)h->n * 4, h->tours, (size_t)h->ld * 4, (size_t)h->n * 4, h->m,
                           cudaMemcpyDeviceToHost));
    if (lens) CK(h, cudaMemcpy(lens, h->lens, (size_t)h->m * 4, cudaMemcpyDeviceToHost));
    return MMAS_OK;
}

mmas_status mmas_get_pheromone(mmas_handle *h, float *tau, float *tau_min, float *tau_max)
{
    if (check_handle(h)) return MMAS_EINVAL;
    DeviceGuard g(h->device);
    mmas_status st = sync_and_check(h);
    if (st != MMAS_OK) return st;
    if (tau)
        CK(h, cudaMemcpy2D(tau, (size_t)h->n * 4, h->tau, (size_t)h->ld * 4, (size_t)h->n * 4, h->n,
                           cudaMemcpyDeviceToHost));
    if (tau_min) *tau_min = h->h_sc->tmin;
    if (tau_max) *tau_max = h->h_sc->tmax;
    return MMAS_OK;
}

mmas_status mmas_set_pheromone(mmas_handle *h, const float *tau, float tau_min, float tau_max)
{
    if (check_handle(h)) return MMAS_EINVAL;
    if (!tau) return fail(h, MMAS_EINVAL, "tau must be non-NULL");
    if (!(tau_min > 0.0f) || !(tau_min <= tau_max) || !std::isfinite(tau_max))
        return fail(h, MMAS_EINVAL, "limits must satisfy 0 < tau_min <= tau_max < inf");
    const size_t nn = (size_t)h->n * h->n;
    for (size_t i = 0; i < nn; ++i)
        if (!(tau[i] > 0.0f) || !std::isfinite(tau[i]))
            return fail(h, MMAS_EINVAL, "pheromone values must be finite and > 0");
    DeviceGuard g(h->device);
    CK(h, cudaMemcpy2DAsync(h->tau, (size_t)h->ld * 4, tau, (size_t)h->n * 4, (size_t)h->n * 4, h->n,
                            cudaMemcpyHostToDevice, h->stream));
    const float lim[2] = {tau_min, tau_max};
    CK(h, cudaMemcpyAsync(&h->sc->tmin, lim, sizeof(lim), cudaMemcpyHostToDevice, h->stream));
    UpdateArgs refresh = h->uargs;
    refresh.evaporate = 0;
    refresh.nbr = nullptr;
    CK(h, launch_update(refresh, h->num_sms, h->stream));
    return MMAS_OK;
}

mmas_status mmas_get_setup(mmas_handle *h, int32_t *dist, float *eta_beta, int32_t *cand,
                           int64_t *nn_len)
{
    if (check_handle(h)) return MMAS_EINVAL;
    DeviceGuard g(h->device);
    mmas_status st = sync_and_check(h);
    if (st != MMAS_OK) return st;
    const size_t row = (size_t)h->n * 4, pitch = (size_t)h->ld * 4;
    if (dist) CK(h, cudaMemcpy2D(dist, row, h->dist, pitch, row, h->n, cudaMemcpyDeviceToHost));
    if (eta_beta) CK(h, cudaMemcpy2D(eta_beta, row, h->eb, pitch, row, h->n, cudaMemcpyDeviceToHost));
    if (cand && h->cl > 0)
        CK(h, cudaMemcpy(cand, h->cand32, (size_t)h->n * h->cl * 4, cudaMemcpyDeviceToHost));
    if (nn_len) *nn_len = h->h_sc->nn_len;
    return MMAS_OK;
}

mmas_status mmas_set_iteration(mmas_handle *h, int32_t it)
{
    if (check_handle(h)) return MMAS_EINVAL;
    if (it < 0) return fail(h, MMAS_EINVAL, "iteration index must be >= 0");
    DeviceGuard g(h->device);
    CK(h, cudaMemcpyAsync(&h->sc->iter, &it, sizeof(it), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return MMAS_OK;
}

mmas_status mmas_stats(mmas_handle *h, mmas_stats_t *out)
{
    if (check_handle(h)) return MMAS_EINVAL;
    if (!out) return fail(h, MMAS_EINVAL, "out must be non-NULL");
    DeviceGuard g(h->device);
    mmas_status st = sync_and_check(h);
    if (st != MMAS_OK) return st;
    const Scalars &s = *h->h_sc;
    out->iterations = s.iterations;
    out->fallback_steps = (int64_t)s.fallback_steps;
    out->nn_len = s.nn_len;
    out->best_len = s.gb_len == INT_MAX ? -1 : s.gb_len;
    out->iter_best_len = s.ib_len;
    out->tau_min = s.tmin;
    out->tau_max = s.tmax;
    out->construct_grid = h->cplan.grid;
    out->construct_block = (h->cplan.cons_warps + h->cplan.gen_warps) * 32;
    out->construct_staged = h->cplan.staged;
    out->construct_smem = (int32_t)h->cplan.smem;
    out->row_pitch = h->ld;
    out->fallback_scans = (int64_t)s.fallback_scans;
    return MMAS_OK;
}

mmas_status mmas_synchronize(mmas_handle *h)
{
    if (check_handle(h)) return MMAS_EINVAL;
    DeviceGuard g(h->device);
    return sync_and_check(h);
}

mmas_status mmas_enable_phase_timing(mmas_handle *h, int32_t enable)
{
    if (check_handle(h)) return MMAS_EINVAL;
    DeviceGuard g(h->device);
    CK(h, cudaStreamSynchronize(h->stream));
    const bool want = enable != 0;
    if (want == h->timing) return MMAS_OK;
    if (want)
        for (cudaEvent_t &e : h->ev)
            if (!e) CK(h, cudaEventCreate(&e));
    h->timing = want;
    h->timed_run = false;
    mmas_status st = capture_iteration(h);
    if (st != MMAS_OK) h->timing = !want;
    return st;
}

mmas_status mmas_phase_times(mmas_handle *h, float *construct_ms, float *rest_ms, float *total_ms)
{
    if (check_handle(h)) return MMAS_EINVAL;
    if (!h->timing || !h->timed_run)
        return fail(h, MMAS_ESTATE, "phase timing is off or no timed iteration has run");
    DeviceGuard g(h->device);
    mmas_status st = sync_and_check(h);
    if (st != MMAS_OK) return st;
    float a = 0.f, b = 0.f;
    CK(h, cudaEventElapsedTime(&a, h->ev[0], h->ev[1]));
    CK(h, cudaEventElapsedTime(&b, h->ev[1], h->ev[2]));
    if (construct_ms) *construct_ms = a;
    if (rest_ms) *rest_ms = b;
    if (total_ms) *total_ms = a + b;
    return MMAS_OK;
}

}  // extern "C"
