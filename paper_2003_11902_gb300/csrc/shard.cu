// One colony's ants sharded over ranks: the per-iteration exchange on device
// buffers (mmas_shard_best_key, mmas_shard_tour, mmas_update_device in
// include/mmas.h).
//
// Within an iteration the ants are independent given the pheromone (MMAS has
// no local pheromone update, Sec. 2.1), so each rank builds its block of the
// colony's ants (draws keyed by the global ant index).  Alg. 1's iteration best
// over all ranks is then one all-reduce (MIN) of a packed 8-byte key
// (length << 32 | global ant) -- the shortest tour, ties to the lower ant --
// and one all-reduce (SUM) of an n-int buffer that only the owner of that ant
// fills; every rank applies the same update to its replica.  All three steps
// here are enqueued on the colony's stream and read or write device memory
// only, so the exchange needs no host round trip: 8 + 4n bytes per rank.
#include <climits>
#include <string>

#include "handle.cuh"

namespace mmas {
namespace {

constexpr int SHARD_THREADS = 1024;

// key = (length << 32) | (ant_offset + k) of the shortest local tour.
__global__ void __launch_bounds__(SHARD_THREADS) k_shard_key(const int32_t *lens, int m, int ant_offset,
                                                             unsigned long long *key)
{
    unsigned long long best = ULLONG_MAX;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const unsigned long long v =
            ((unsigned long long)(uint32_t)lens[k] << 32) | (uint32_t)(ant_offset + k);
        best = v < best ? v : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xFFFFFFFFu, best, o);
        best = x < best ? x : best;
    }
    __shared__ unsigned long long s[SHARD_THREADS / 32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = s[w] < best ? s[w] : best;
        *key = best;
    }
}

// The tour of the key's ant when this colony builds it, else zeros.
__global__ void k_shard_tour(const unsigned long long *key, const int32_t *tours, int n, int m, int ld,
                             int ant_offset, int32_t *out)
{
    const long long local = (long long)(uint32_t)(*key & 0xFFFFFFFFull) - ant_offset;
    const bool mine = local >= 0 && local < m;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = mine ? tours[(size_t)local * ld + i] : 0;
}

// Check that `tour` is a permutation of 0..n-1 and the key's length positive;
// then hand both to the update (ext_tour, ext_len), else raise ERR_BAD_TOUR and
// set *bad_out, which makes the update's steps do nothing.  One CTA; a bitmap
// of n bits in shared memory.
__global__ void __launch_bounds__(SHARD_THREADS) k_shard_accept(const int32_t *tour, const unsigned long long *key,
                                                                int n, int32_t *ext_tour, int32_t *ext_len,
                                                                uint32_t *bad_out, uint32_t *err)
{
    extern __shared__ uint32_t seen[];
    __shared__ int bad;
    const int words = (n + 31) >> 5;
    for (int w = threadIdx.x; w < words; w += blockDim.x) seen[w] = 0u;
    if (threadIdx.x == 0) {
        const unsigned long long k = *key;
        bad = (k >> 32) == 0 || (k >> 32) > (unsigned long long)INT_MAX;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int v = tour[i];
        if (v < 0 || v >= n) {
            bad = 1;
            continue;
        }
        if (atomicOr(&seen[v >> 5], 1u << (v & 31)) & (1u << (v & 31))) bad = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) *bad_out = bad ? 1u : 0u;  // the update steps that follow read it
    if (bad) {
        if (threadIdx.x == 0) atomicOr(err, ERR_BAD_TOUR);
        return;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) ext_tour[i] = tour[i];
    if (threadIdx.x == 0) *ext_len = (int32_t)(*key >> 32);
}

mmas_status shard_fail(mmas_handle *h, mmas_status st, const std::string &msg)
{
    h->err = msg;
    return st;
}

}  // namespace
}  // namespace mmas

using namespace mmas;

#define SCK(h, call)                                                                        \
    do {                                                                                    \
        const cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) return shard_fail((h), MMAS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace {
struct ShardDevice {
    int prev = -1;
    explicit ShardDevice(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~ShardDevice()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
}  // namespace

extern "C" {

mmas_status mmas_shard_best_key(mmas_handle *h, int64_t *d_key)
{
    if (!h) return MMAS_EINVAL;
    if (!d_key) return shard_fail(h, MMAS_EINVAL, "d_key must be a device pointer");
    ShardDevice g(h->device);
    k_shard_key<<<1, SHARD_THREADS, 0, h->stream>>>(h->lens, h->m, h->p.ant_offset,
                                                    reinterpret_cast<unsigned long long *>(d_key));
    SCK(h, cudaGetLastError());
    return MMAS_OK;
}

mmas_status mmas_shard_tour(mmas_handle *h, const int64_t *d_key, int32_t *d_tour)
{
    if (!h) return MMAS_EINVAL;
    if (!d_key || !d_tour) return shard_fail(h, MMAS_EINVAL, "d_key and d_tour must be device pointers");
    ShardDevice g(h->device);
    const int blocks = (h->n + 255) / 256;
    k_shard_tour<<<blocks, 256, 0, h->stream>>>(reinterpret_cast<const unsigned long long *>(d_key), h->tours,
                                                 h->n, h->m, h->ld, h->p.ant_offset, d_tour);
    SCK(h, cudaGetLastError());
    return MMAS_OK;
}

mmas_status mmas_update_device(mmas_handle *h, const int32_t *d_tour, const int64_t *d_key)
{
    if (!h) return MMAS_EINVAL;
    if (!d_key || !d_tour) return shard_fail(h, MMAS_EINVAL, "d_tour and d_key must be device pointers");
    ShardDevice g(h->device);
    const size_t bitmap = (size_t)((h->n + 31) >> 5) * sizeof(uint32_t);
    k_shard_accept<<<1, SHARD_THREADS, bitmap, h->stream>>>(d_tour, reinterpret_cast<const unsigned long long *>(d_key),
                                                            h->n, h->ext_tour, h->ext_len, h->ext_bad,
                                                            &h->sc->err);
    SCK(h, cudaGetLastError());
    BestArgs b = h->bargs;
    b.m = 1;
    b.lens = h->ext_len;
    b.tours = h->ext_tour;
    b.advance = 1;  // one sharded iteration ends here, as a whole iteration does
    b.skip = h->ext_bad;
    UpdateArgs u = h->uargs;
    u.skip = h->ext_bad;
    SCK(h, launch_best(b, h->stream));
    SCK(h, launch_update(u, h->num_sms, h->stream));
    return MMAS_OK;
}

}  // extern "C"
