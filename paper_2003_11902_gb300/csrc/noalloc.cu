// Allocation-free tour scoring: mmas_score_tours_noalloc (see include/mmas.h).
//
// Some callers cannot let a library allocate device memory: serving loops that
// must not stall on cudaMalloc/cudaFree (which synchronise the device), and
// frameworks whose caching allocator owns the whole memory budget.  This entry
// point scores tours that already sit in device memory using only buffers the
// caller passes plus a small scratch array that lives in this file as a
// file-scope __device__ variable, so no call ever allocates.
//
// The scratch holds one partial minimum per CTA and a completion counter.
// Every GPU that loads the library keeps it (NOALLOC_MAX_CTAS * 8 + 256 bytes)
// until the process exits.  Every call shares it: calls whose GPU work overlaps
// (different streams, no ordering between them) race on it.
#include <climits>
#include <cstdint>
#include <mutex>
#include <string>

#include "distance.cuh"
#include "internal.cuh"
#include "mmas.h"

namespace {

constexpr int NOALLOC_MAX_CTAS = 4096;
constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr int NOALLOC_THREADS = 256;

struct NoallocScratch {
    unsigned long long partial[NOALLOC_MAX_CTAS];  // per-CTA (length << 32 | ant) minimum
    unsigned int done;                              // CTAs finished in the current call
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

std::mutex g_setup_mutex;
NoallocScratch *g_scratch_addr[NOALLOC_MAX_DEVICES] = {};

// One CTA per ant (looping when m exceeds the grid); each thread sums four
// consecutive edges per round with exact TSPLIB distances from coordinates.
// Each CTA keeps its smallest (length, ant) key; the last CTA to finish reduces
// the partial minima into best[0] = length, best[1] = ant (ties -> lower ant)
// and zeroes the completion counter for the next call.
__global__ void __launch_bounds__(NOALLOC_THREADS)
    k_score_noalloc(const int32_t *__restrict__ tours, int32_t m, int32_t n, int32_t pitch,
                    const int2 *__restrict__ xy, int32_t *__restrict__ lens,
                    int32_t *__restrict__ best, NoallocScratch *scratch)
{
    __shared__ int red[NOALLOC_THREADS / 32];
    __shared__ unsigned long long redk[NOALLOC_THREADS / 32];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = NOALLOC_THREADS / 32;
    unsigned long long cta_min = ~0ull;
    for (int ant = blockIdx.x; ant < m; ant += gridDim.x) {
        const int32_t *tr = tours + (size_t)ant * pitch;
        int part = 0;
        for (int t0 = 4 * tid; t0 < n; t0 += 4 * NOALLOC_THREADS) {
            int node[5];
#pragma unroll
            for (int e = 0; e < 5; ++e) node[e] = t0 + e < n ? tr[t0 + e] : tr[0];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (t0 + e < n) part += mmas::euc2d_exact(__ldg(xy + node[e]), __ldg(xy + node[e + 1]));
        }
        part = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)part);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (tid == 0) {
            int sum = 0;
            for (int i = 0; i < nwarps; ++i) sum += red[i];
            lens[ant] = sum;
            const unsigned long long key = ((unsigned long long)(uint32_t)sum << 32) | (uint32_t)ant;
            cta_min = key < cta_min ? key : cta_min;
        }
        __syncthreads();
    }
    if (tid == 0) scratch->partial[blockIdx.x] = cta_min;
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&scratch->done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long v = ~0ull;
    for (int i = tid; i < (int)gridDim.x; i += NOALLOC_THREADS) {
        const unsigned long long k = __ldcg(scratch->partial + i);
        v = k < v ? k : v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = w < v ? w : v;
    }
    if (lane == 0) redk[warp] = v;
    __syncthreads();
    if (tid == 0) {
        unsigned long long b = redk[0];
        for (int i = 1; i < nwarps; ++i) b = redk[i] < b ? redk[i] : b;
        best[0] = (int32_t)(b >> 32);
        best[1] = (int32_t)(b & 0xFFFFFFFFull);
        scratch->done = 0;
    }
}

// Device address of the scratch on the current device, looked up once per
// device with that device current.
cudaError_t scratch_address(NoallocScratch **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<NoallocScratch *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" mmas_status mmas_score_tours_noalloc(const int32_t *d_tours, int32_t m, int32_t n,
                                                int32_t pitch, const int32_t *d_xy,
                                                int32_t *d_lens, int32_t *d_best, void *stream)
{
    using mmas::set_thread_error;
    if (!d_tours || !d_xy || !d_lens || !d_best) {
        set_thread_error("mmas_score_tours_noalloc: every buffer must be non-NULL");
        return MMAS_EINVAL;
    }
    if (m < 1 || m > MMAS_NOALLOC_MAX_ANTS) {
        set_thread_error("mmas_score_tours_noalloc: m must be in [1, MMAS_NOALLOC_MAX_ANTS = 1048576]");
        return MMAS_EINVAL;
    }
    if (n < 3 || n > 65535 || pitch < n) {
        set_thread_error("mmas_score_tours_noalloc: need 3 <= n <= 65535 and pitch >= n");
        return MMAS_EINVAL;
    }
    // the kernel reads coordinates as 8-byte pairs and the rest as 4-byte words
    if ((reinterpret_cast<uintptr_t>(d_xy) & 7u) != 0 || (reinterpret_cast<uintptr_t>(d_tours) & 3u) != 0 ||
        (reinterpret_cast<uintptr_t>(d_lens) & 3u) != 0 || (reinterpret_cast<uintptr_t>(d_best) & 3u) != 0) {
        set_thread_error("mmas_score_tours_noalloc: d_xy must be 8-byte aligned and d_tours, d_lens, d_best "
                         "4-byte aligned");
        return MMAS_EINVAL;
    }
    NoallocScratch *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        set_thread_error(std::string("mmas_score_tours_noalloc: cudaGetSymbolAddress: ") +
                         cudaGetErrorString(e));
        return MMAS_ECUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the counter must start at zero even if an earlier call was interrupted
    e = cudaMemsetAsync(&scratch->done, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        const int grid = m < NOALLOC_MAX_CTAS ? m : NOALLOC_MAX_CTAS;
        k_score_noalloc<<<grid, NOALLOC_THREADS, 0, s>>>(d_tours, m, n, pitch,
                                                        reinterpret_cast<const int2 *>(d_xy),
                                                        d_lens, d_best, scratch);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_thread_error(std::string("mmas_score_tours_noalloc: ") + cudaGetErrorString(e));
        return MMAS_ECUDA;
    }
    return MMAS_OK;
}
