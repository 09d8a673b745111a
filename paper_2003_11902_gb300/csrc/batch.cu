// Batched colonies behind the mmas_batch_* C ABI (include/mmas.h).
//
// A batch owns B ordinary colonies (built by mmas_create with seed + b on the
// batch's stream, so set-up, validation and every per-colony buffer are the
// single-colony ones) plus the tables the three batched launches read:
//   cargs / sargs / uargs   per-colony construction, scoring, update arguments
//   chunks                  (colony, first ant, count) units of construction,
//                           ordered by decreasing n (longest tours first)
//   ant_colony / ant_base   global ant -> colony, and each colony's first ant
//   row_colony / row_base   global row -> colony, and each colony's first row
// One iteration of all colonies is a CUDA graph: reset the chunk counter,
// construct, score (with each colony's best / limits in its last CTA), update.
#include <algorithm>
#include <climits>
#include <new>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace mmas;

struct mmas_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    size_t smem_optin = 0, smem_per_sm = 0, smem_reserved = 0;
    std::vector<mmas_handle *> col;
    bool xy = true, alpha1 = true;
    int total_ants = 0, total_rows = 0, max_n = 0;

    ConstructArgs *d_cargs = nullptr;
    ScoreArgs *d_sargs = nullptr;
    UpdateArgs *d_uargs = nullptr;
    int32_t *d_ant_colony = nullptr, *d_ant_base = nullptr;
    int32_t *d_row_colony = nullptr, *d_row_base = nullptr;
    BatchChunk *d_chunks = nullptr;
    int nchunks = 0, chunk_cap = 0;
    unsigned *d_counter = nullptr;
    Scalars **d_scs = nullptr;       // each colony's scalar block
    int32_t *d_best = nullptr;       // gathered global best lengths [count]
    unsigned long long *d_gather = nullptr;  // {err bits, fallback sum}
    int32_t *h_best = nullptr;       // pinned mirrors
    unsigned long long *h_gather = nullptr;

    mmas_batch_config cfg{12, 1};
    size_t cta_smem = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool timing = false, timed_run = false;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    std::string err;
};

namespace {

thread_local std::string tl_batch_error;

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

mmas_status bfail(mmas_batch *b, mmas_status st, const std::string &msg)
{
    if (b)
        b->err = msg;
    else
        tl_batch_error = msg;
    return st;
}

#define BCK(b, call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? MMAS_ENOMEM : MMAS_ECUDA,   \
                         std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

// Global best length of every colony, the OR of their error bits and the sum
// of their fallback counters, gathered in one launch.
__global__ void k_batch_gather(Scalars *const *scs, int count, int32_t *best,
                               unsigned long long *out)
{
    unsigned long long errs = 0, fb = 0;
    for (int b = threadIdx.x; b < count; b += blockDim.x) {
        const Scalars *s = scs[b];
        best[b] = s->gb_len == INT_MAX ? -1 : s->gb_len;
        errs |= s->err;
        fb += s->fallback_steps;
    }
    for (int o = 16; o > 0; o >>= 1) {
        errs |= __shfl_xor_sync(0xFFFFFFFFu, errs, o);
        fb += __shfl_xor_sync(0xFFFFFFFFu, fb, o);
    }
    __shared__ unsigned long long se[32], sf[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        se[warp] = errs;
        sf[warp] = fb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long e = 0, f = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            e |= se[w];
            f += sf[w];
        }
        out[0] = e;
        out[1] = f;
    }
}

__global__ void k_batch_reset_fallbacks(Scalars *const *scs, int count)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x) {
        scs[b]->fallback_steps = 0;
        scs[b]->fallback_scans = 0;
    }
}

void free_batch(mmas_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    void *bufs[] = {b->d_cargs, b->d_sargs, b->d_uargs, b->d_ant_colony, b->d_ant_base,
                    b->d_row_colony, b->d_row_base, b->d_chunks, b->d_counter, b->d_scs,
                    b->d_best, b->d_gather};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (b->h_best) cudaFreeHost(b->h_best);
    if (b->h_gather) cudaFreeHost(b->h_gather);
    for (mmas_handle *h : b->col) mmas_destroy(h);
    b->col.clear();
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

// Synchronise, gather every colony's best length, error bits and fallbacks.
mmas_status gather(mmas_batch *b)
{
    const int count = (int)b->col.size();
    k_batch_gather<<<1, 256, 0, b->stream>>>(b->d_scs, count, b->d_best, b->d_gather);
    BCK(b, cudaGetLastError());
    BCK(b, cudaMemcpyAsync(b->h_best, b->d_best, (size_t)count * 4, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaMemcpyAsync(b->h_gather, b->d_gather, 16, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    const unsigned long long e = b->h_gather[0];
    if (e & ERR_STAGE_TIMEOUT)
        return bfail(b, MMAS_ETIMEOUT, "a candidate-table copy did not complete in time");
    if (e & ERR_NO_UNVISITED) return bfail(b, MMAS_ESTATE, "a selection found no unvisited node");
    return MMAS_OK;
}

// Every colony has n <= 2048: the batched construction's narrow variant, whose
// register budget lets 16 warps share an SM (12 otherwise).
bool narrow(const mmas_batch *b) { return b->max_n <= 2048; }
int max_warps(const mmas_batch *b) { return narrow(b) ? 16 : 12; }

// Shared memory per construction CTA for `ctas` CTAs per SM.
size_t cta_smem_for(const mmas_batch *b, int ctas)
{
    const size_t static_smem = 1024;  // the kernel's own shared variables, rounded up
    size_t per = b->smem_per_sm / (size_t)ctas;
    per = per > b->smem_reserved + static_smem ? per - b->smem_reserved - static_smem : 0;
    per &= ~size_t(127);
    return std::min(per, b->smem_optin - static_smem);
}

mmas_status check_config(mmas_batch *b, const mmas_batch_config &c, size_t *smem)
{
    const int wmax = max_warps(b);
    if (c.warps_per_cta < 1 || c.warps_per_cta > wmax || c.ctas_per_sm < 1 || c.ctas_per_sm > 4)
        return bfail(b, MMAS_EINVAL, wmax == 16 ? "warps_per_cta must be in 1..16 and ctas_per_sm in 1..4"
                                                : "warps_per_cta must be in 1..12 (a colony has n > 2048) "
                                                  "and ctas_per_sm in 1..4");
    if (c.warps_per_cta * c.ctas_per_sm > wmax)
        return bfail(b, MMAS_EINVAL, "warps_per_cta x ctas_per_sm exceeds the construction warps one "
                                     "SM's registers hold (16, or 12 with a colony of n > 2048)");
    const size_t s = cta_smem_for(b, c.ctas_per_sm);
    // the shared-memory tabus of the largest colony must fit when its table does not
    const size_t masks =
        b->max_n > 1024 ? (size_t)c.warps_per_cta * ((b->max_n + 31) / 32) * sizeof(uint32_t) : 0;
    if (masks > s) return bfail(b, MMAS_EINVAL, "the tabu lists of the largest colony do not fit");
    *smem = s;
    return MMAS_OK;
}

// Chunks of up to `w` ants, colonies by decreasing n (ties: lower index).
mmas_status build_chunks(mmas_batch *b, int w)
{
    std::vector<int> order(b->col.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->col[x]->n > b->col[y]->n; });
    std::vector<BatchChunk> ch;
    for (int c : order)
        for (int f = 0; f < b->col[c]->m; f += w)
            ch.push_back(BatchChunk{c, f, std::min(w, b->col[c]->m - f)});
    if ((int)ch.size() > b->chunk_cap) {
        if (b->d_chunks) cudaFree(b->d_chunks);
        b->d_chunks = nullptr;
        BCK(b, device_malloc(&b->d_chunks, ch.size() * sizeof(BatchChunk)));
        b->chunk_cap = (int)ch.size();
    }
    BCK(b, cudaMemcpyAsync(b->d_chunks, ch.data(), ch.size() * sizeof(BatchChunk),
                           cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    b->nchunks = (int)ch.size();
    return MMAS_OK;
}

mmas_status enqueue_construct(mmas_batch *b, cudaStream_t s)
{
    BCK(b, cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), s));
    BCK(b, launch_construct_batch(b->d_cargs, b->d_chunks, b->nchunks, b->d_counter,
                                  b->num_sms * b->cfg.ctas_per_sm, b->cfg.warps_per_cta, b->cta_smem,
                                  narrow(b), s));
    return MMAS_OK;
}

mmas_status capture(mmas_batch *b)
{
    cudaStream_t cs;
    BCK(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess && b->timing) e = cudaEventRecordWithFlags(b->ev[0], cs, cudaEventRecordExternal);
    mmas_status st = MMAS_OK;
    if (e == cudaSuccess) st = enqueue_construct(b, cs);
    if (e == cudaSuccess && st == MMAS_OK && b->timing)
        e = cudaEventRecordWithFlags(b->ev[1], cs, cudaEventRecordExternal);
    if (e == cudaSuccess && st == MMAS_OK)
        e = launch_score_batch(b->d_sargs, b->d_ant_colony, b->d_ant_base, b->total_ants, b->xy, cs);
    if (e == cudaSuccess && st == MMAS_OK)
        e = launch_update_batch(b->d_uargs, b->d_row_colony, b->d_row_base, b->total_rows, b->alpha1, cs);
    if (e == cudaSuccess && st == MMAS_OK && b->timing)
        e = cudaEventRecordWithFlags(b->ev[2], cs, cudaEventRecordExternal);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st != MMAS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, MMAS_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return bfail(b, MMAS_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    }
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph = g;
    b->gexec = ge;
    return MMAS_OK;
}

// Make c the construction launch shape (chunks, shared memory) without
// re-recording the graph.
mmas_status apply_config(mmas_batch *b, const mmas_batch_config &c)
{
    size_t smem = 0;
    mmas_status st = check_config(b, c, &smem);
    if (st != MMAS_OK) return st;
    st = build_chunks(b, c.warps_per_cta);
    if (st != MMAS_OK) return st;
    BCK(b, prepare_construct_batch(smem, narrow(b)));
    b->cfg = c;
    b->cta_smem = smem;
    return MMAS_OK;
}

mmas_status create_batch(mmas_batch *b, const mmas_instance *insts, int count, const mmas_params &p)
{
    cudaDeviceProp prop;
    BCK(b, cudaGetDeviceProperties(&prop, b->device));
    b->num_sms = prop.multiProcessorCount;
    b->smem_optin = prop.sharedMemPerBlockOptin;
    b->smem_per_sm = prop.sharedMemPerMultiprocessor;
    b->smem_reserved = prop.reservedSharedMemPerBlock;
    if (p.stream) {
        b->stream = static_cast<cudaStream_t>(p.stream);
    } else {
        BCK(b, cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    b->col.reserve(count);
    for (int c = 0; c < count; ++c) {
        mmas_params pc = p;
        pc.seed = p.seed + (uint64_t)c;
        pc.stream = b->stream;
        mmas_handle *h = nullptr;
        const mmas_status st = mmas_create(&insts[c], &pc, &h);
        if (st != MMAS_OK)
            return bfail(b, st, "colony " + std::to_string(c) + ": " + mmas_last_error(nullptr));
        b->col.push_back(h);
        b->max_n = std::max(b->max_n, h->n);
    }
    const int B = count;
    std::vector<ConstructArgs> ca(B);
    std::vector<ScoreArgs> sa(B);
    std::vector<UpdateArgs> ua(B);
    std::vector<int32_t> ant_colony, ant_base(B), row_colony, row_base(B);
    std::vector<Scalars *> scs(B);
    for (int c = 0; c < B; ++c) {
        const mmas_handle *h = b->col[c];
        ca[c] = h->cargs;
        sa[c] = h->sargs;
        sa[c].best = 1;
        ua[c] = h->uargs;
        // no extra list for the greedy fallback in batched runs: its upkeep
        // costs the pass more than the short runs of many colonies gain
        ua[c].xhot = nullptr;
        scs[c] = h->sc;
        ant_base[c] = (int32_t)ant_colony.size();
        for (int k = 0; k < h->m; ++k) ant_colony.push_back(c);
        row_base[c] = (int32_t)row_colony.size();
        for (int i = 0; i < h->n; ++i) row_colony.push_back(c);
    }
    b->total_ants = (int)ant_colony.size();
    b->total_rows = (int)row_colony.size();
    b->alpha1 = p.alpha == 1.0f;
    auto upload = [&](auto **dst, const auto &v) -> mmas_status {
        const size_t bytes = v.size() * sizeof(v[0]);
        BCK(b, device_malloc(reinterpret_cast<void **>(dst), bytes));
        BCK(b, cudaMemcpyAsync(*dst, v.data(), bytes, cudaMemcpyHostToDevice, b->stream));
        return MMAS_OK;
    };
    mmas_status st;
    if ((st = upload(&b->d_cargs, ca)) != MMAS_OK) return st;
    if ((st = upload(&b->d_sargs, sa)) != MMAS_OK) return st;
    if ((st = upload(&b->d_uargs, ua)) != MMAS_OK) return st;
    if ((st = upload(&b->d_ant_colony, ant_colony)) != MMAS_OK) return st;
    if ((st = upload(&b->d_ant_base, ant_base)) != MMAS_OK) return st;
    if ((st = upload(&b->d_row_colony, row_colony)) != MMAS_OK) return st;
    if ((st = upload(&b->d_row_base, row_base)) != MMAS_OK) return st;
    if ((st = upload(&b->d_scs, scs)) != MMAS_OK) return st;
    BCK(b, device_malloc(&b->d_counter, sizeof(unsigned)));
    BCK(b, device_malloc(&b->d_best, (size_t)B * sizeof(int32_t)));
    BCK(b, device_malloc(&b->d_gather, 2 * sizeof(unsigned long long)));
    BCK(b, cudaMallocHost(&b->h_best, (size_t)B * sizeof(int32_t)));
    BCK(b, cudaMallocHost(&b->h_gather, 2 * sizeof(unsigned long long)));
    BCK(b, cudaStreamSynchronize(b->stream));
    mmas_batch_config c0{max_warps(b), 1};
    if ((st = apply_config(b, c0)) != MMAS_OK) return st;
    if ((st = capture(b)) != MMAS_OK) return st;
    return gather(b);
}

mmas_status check_batch(mmas_batch *b)
{
    if (!b) return bfail(nullptr, MMAS_EINVAL, "batch is NULL");
    return MMAS_OK;
}

mmas_status check_colony(mmas_batch *b, int32_t c)
{
    if (c < 0 || c >= (int32_t)b->col.size()) return bfail(b, MMAS_EINVAL, "colony index out of range");
    return MMAS_OK;
}

}  // namespace

extern "C" {

mmas_status mmas_batch_create(const mmas_instance *instances, int32_t count, const mmas_params *params,
                              mmas_batch **out)
{
    if (!out) return bfail(nullptr, MMAS_EINVAL, "out must be non-NULL");
    *out = nullptr;
    tl_batch_error.clear();
    if (!instances || !params || count < 1)
        return bfail(nullptr, MMAS_EINVAL, "instances and params must be non-NULL and count >= 1");
    const mmas_params &p = *params;
    if (p.cl < 1 || p.cl > 32) return bfail(nullptr, MMAS_EINVAL, "batched colonies need 1 <= cl <= 32");
    if (p.ls != 0) return bfail(nullptr, MMAS_EINVAL, "batched colonies run without local search (ls = 0)");
    if (p.ant_offset != 0) return bfail(nullptr, MMAS_EINVAL, "batched colonies need ant_offset = 0");
    const bool xy = instances[0].xy != nullptr;
    for (int c = 0; c < count; ++c)
        if ((instances[c].xy != nullptr) != xy)
            return bfail(nullptr, MMAS_EINVAL,
                         "every instance must have coordinates, or every instance a matrix");
    for (int c = 0; c < count; ++c) {
        mmas_params pc = p;
        pc.seed = p.seed + (uint64_t)c;
        if (validate_colony(&instances[c], &pc) != MMAS_OK)
            return bfail(nullptr, MMAS_EINVAL,
                         "colony " + std::to_string(c) + ": " + mmas_last_error(nullptr));
    }
    mmas_batch *b = new (std::nothrow) mmas_batch();
    if (!b) return bfail(nullptr, MMAS_ENOMEM, "host allocation failed");
    b->device = p.device;
    b->xy = xy;
    DeviceGuard g(b->device);
    const mmas_status st = create_batch(b, instances, count, p);
    if (st != MMAS_OK) {
        tl_batch_error = b->err;
        if (b->stream) cudaStreamSynchronize(b->stream);
        free_batch(b);
        delete b;
        return st;
    }
    *out = b;
    return MMAS_OK;
}

mmas_status mmas_batch_iterate(mmas_batch *b, int32_t k)
{
    if (check_batch(b)) return MMAS_EINVAL;
    if (k < 0) return bfail(b, MMAS_EINVAL, "k must be >= 0");
    DeviceGuard g(b->device);
    for (int32_t i = 0; i < k; ++i) BCK(b, cudaGraphLaunch(b->gexec, b->stream));
    if (k > 0 && b->timing) b->timed_run = true;
    return MMAS_OK;
}

mmas_status mmas_batch_best_tour(mmas_batch *b, int32_t colony, int32_t *tour_out, int32_t *len_out)
{
    if (check_batch(b) || check_colony(b, colony)) return MMAS_EINVAL;
    DeviceGuard g(b->device);
    const mmas_status st = mmas_best_tour(b->col[colony], tour_out, len_out);
    if (st != MMAS_OK) return bfail(b, st, mmas_last_error(b->col[colony]));
    return MMAS_OK;
}

mmas_status mmas_batch_best_lengths(mmas_batch *b, int32_t *lens_out)
{
    if (check_batch(b)) return MMAS_EINVAL;
    if (!lens_out) return bfail(b, MMAS_EINVAL, "lens_out must be non-NULL");
    DeviceGuard g(b->device);
    const mmas_status st = gather(b);
    if (st != MMAS_OK) return st;
    std::copy(b->h_best, b->h_best + b->col.size(), lens_out);
    return MMAS_OK;
}

mmas_status mmas_batch_get_tours(mmas_batch *b, int32_t colony, int32_t *tours, int32_t *lens)
{
    if (check_batch(b) || check_colony(b, colony)) return MMAS_EINVAL;
    DeviceGuard g(b->device);
    const mmas_status st = mmas_get_tours(b->col[colony], tours, lens);
    if (st != MMAS_OK) return bfail(b, st, mmas_last_error(b->col[colony]));
    return MMAS_OK;
}

mmas_status mmas_batch_colony(mmas_batch *b, int32_t colony, mmas_handle **out)
{
    if (check_batch(b) || check_colony(b, colony)) return MMAS_EINVAL;
    if (!out) return bfail(b, MMAS_EINVAL, "out must be non-NULL");
    *out = b->col[colony];
    return MMAS_OK;
}

mmas_status mmas_batch_set_config(mmas_batch *b, const mmas_batch_config *cfg)
{
    if (check_batch(b)) return MMAS_EINVAL;
    if (!cfg) return bfail(b, MMAS_EINVAL, "cfg must be non-NULL");
    DeviceGuard g(b->device);
    BCK(b, cudaStreamSynchronize(b->stream));
    const mmas_batch_config prev = b->cfg;
    mmas_status st = apply_config(b, *cfg);
    if (st != MMAS_OK) {
        const std::string msg = b->err;
        apply_config(b, prev);
        return bfail(b, st, msg);
    }
    return capture(b);
}

mmas_status mmas_batch_get_config(mmas_batch *b, mmas_batch_config *cfg)
{
    if (check_batch(b)) return MMAS_EINVAL;
    if (!cfg) return bfail(b, MMAS_EINVAL, "cfg must be non-NULL");
    *cfg = b->cfg;
    return MMAS_OK;
}

mmas_status mmas_batch_autotune(mmas_batch *b, int32_t reps, mmas_batch_config *chosen)
{
    if (check_batch(b)) return MMAS_EINVAL;
    if (reps < 1) return bfail(b, MMAS_EINVAL, "reps must be >= 1");
    DeviceGuard g(b->device);
    BCK(b, cudaStreamSynchronize(b->stream));
    static const mmas_batch_config wide[] = {{12, 1}, {8, 1}, {6, 2}, {4, 3}, {3, 4}, {10, 1}};
    static const mmas_batch_config narrow_cands[] = {{16, 1}, {14, 1}, {12, 1}, {8, 2}, {4, 4}, {5, 3}};
    const std::vector<mmas_batch_config> cands =
        narrow(b) ? std::vector<mmas_batch_config>(std::begin(narrow_cands), std::end(narrow_cands))
                  : std::vector<mmas_batch_config>(std::begin(wide), std::end(wide));
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    mmas_batch_config best = b->cfg;
    float best_ms = -1.0f;
    mmas_status st = MMAS_OK;
    for (const mmas_batch_config &c : cands) {
        size_t smem = 0;
        if (check_config(b, c, &smem) != MMAS_OK) continue;  // not feasible for these colonies
        if ((st = apply_config(b, c)) != MMAS_OK) break;
        if ((st = enqueue_construct(b, b->stream)) != MMAS_OK) break;  // warm-up
        std::vector<float> t;
        for (int r = 0; r < reps && st == MMAS_OK; ++r) {
            cudaEventRecord(e0, b->stream);
            st = enqueue_construct(b, b->stream);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = bfail(b, MMAS_ECUDA, "autotune timing failed");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t.push_back(ms);
        }
        if (st != MMAS_OK) break;
        std::nth_element(t.begin(), t.begin() + t.size() / 2, t.end());
        const float med = t[t.size() / 2];
        if (best_ms < 0.0f || med < best_ms) {
            best_ms = med;
            best = c;
        }
    }
    b->err.clear();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MMAS_OK) return st;
    if ((st = apply_config(b, best)) != MMAS_OK) return st;
    k_batch_reset_fallbacks<<<(int)(b->col.size() + 255) / 256, 256, 0, b->stream>>>(
        b->d_scs, (int)b->col.size());
    BCK(b, cudaGetLastError());
    if ((st = capture(b)) != MMAS_OK) return st;
    if ((st = gather(b)) != MMAS_OK) return st;
    if (chosen) *chosen = best;
    return MMAS_OK;
}

mmas_status mmas_batch_synchronize(mmas_batch *b)
{
    if (check_batch(b)) return MMAS_EINVAL;
    DeviceGuard g(b->device);
    return gather(b);
}

mmas_status mmas_batch_enable_phase_timing(mmas_batch *b, int32_t enable)
{
    if (check_batch(b)) return MMAS_EINVAL;
    DeviceGuard g(b->device);
    BCK(b, cudaStreamSynchronize(b->stream));
    const bool want = enable != 0;
    if (want == b->timing) return MMAS_OK;
    if (want)
        for (cudaEvent_t &e : b->ev)
            if (!e) BCK(b, cudaEventCreate(&e));
    b->timing = want;
    b->timed_run = false;
    const mmas_status st = capture(b);
    if (st != MMAS_OK) b->timing = !want;
    return st;
}

mmas_status mmas_batch_phase_times(mmas_batch *b, float *construct_ms, float *rest_ms, float *total_ms)
{
    if (check_batch(b)) return MMAS_EINVAL;
    if (!b->timing || !b->timed_run)
        return bfail(b, MMAS_ESTATE, "phase timing is off or no timed iteration has run");
    DeviceGuard g(b->device);
    const mmas_status st = gather(b);
    if (st != MMAS_OK) return st;
    float x = 0.f, y = 0.f;
    BCK(b, cudaEventElapsedTime(&x, b->ev[0], b->ev[1]));
    BCK(b, cudaEventElapsedTime(&y, b->ev[1], b->ev[2]));
    if (construct_ms) *construct_ms = x;
    if (rest_ms) *rest_ms = y;
    if (total_ms) *total_ms = x + y;
    return MMAS_OK;
}

mmas_status mmas_batch_fallback_steps(mmas_batch *b, int64_t *out)
{
    if (check_batch(b)) return MMAS_EINVAL;
    if (!out) return bfail(b, MMAS_EINVAL, "out must be non-NULL");
    DeviceGuard g(b->device);
    const mmas_status st = gather(b);
    if (st != MMAS_OK) return st;
    *out = (int64_t)b->h_gather[1];
    return MMAS_OK;
}

void mmas_batch_destroy(mmas_batch *b)
{
    if (!b) return;
    DeviceGuard g(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
}

const char *mmas_batch_last_error(const mmas_batch *b)
{
    return b ? b->err.c_str() : tl_batch_error.c_str();
}

}  // extern "C"
