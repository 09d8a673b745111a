// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05 / UMMA),
// FP32 accumulation in tensor memory, for the learned edge prior:
//
//   D[M x N] = act(A[M x K] * B[N x K]^T + bias[N])   (+ optional residual R[M x N])
//
// A and B are bf16 and K-major (row-major with K contiguous, leading dimension
// lda / ldb elements); D is fp32 or bf16, row-major; N is 64 or 128; M and K
// are arbitrary (tiles are guarded, missing rows and columns read as zero).
//
// One CTA of four warps computes a 128 x N tile of D.  Per 64-wide K block the
// CTA copies the A tile (128 x 64) and B tile (N x 64) into shared memory in the
// canonical K-major 128-byte-swizzled layout (rows of 128 bytes, 8-row atoms of
// 1 KB, the 16-byte chunk c of row r stored at chunk c ^ (r mod 8)); one thread
// issues four MMAs (K = 16 each, the descriptor start advanced by 32 bytes)
// and commits them to the stage's mbarrier.  Two stages: block i + 1 is copied
// while the MMAs of block i run, and a stage is rewritten only after its MMAs
// completed (bounded waits).  Split-K (launch_gemm_bf16_splitk): CTAs along
// grid.y take disjoint ranges of K blocks and atomically add their fp32 tiles
// into a zeroed output, for the long-K products (K = n) of the weight gradients.  The accumulator lives in TMEM (N columns); the
// epilogue reads it with tcgen05.ld (warp w owns rows 32w .. 32w+31), applies
// bias, residual and ReLU, and stores D.
#include <cuda_bf16.h>

#include <string>

#include "internal.cuh"
#include "mmas.h"

namespace mmas {
namespace {

constexpr int TM = 128;  // rows of D per CTA
constexpr int TK = 64;   // K per shared-memory block (one 128-byte swizzle row)
constexpr unsigned long long MMA_LIMIT_NS = 2000000000ull;  // 2 s

struct GemmArgs {
    const __nv_bfloat16 *a;
    const __nv_bfloat16 *b;
    const float *bias;      // [N] or nullptr
    const float *resid;     // [M][ldr] fp32 or nullptr
    float *d32;             // fp32 output or nullptr
    __nv_bfloat16 *d16;     // bf16 output or nullptr
    int m, n, k, lda, ldb, ldd, ldr, relu;
    uint32_t *err;          // set on an MMA-completion timeout
    int kb_per_split;       // K blocks per CTA along grid.y (split-K)
    int accumulate;         // 1: atomically add the fp32 tile into d32 (split-K), no epilogue ops
};

// Canonical UMMA shared-memory descriptor (tcgen05): start address >> 4,
// leading byte offset (unused for swizzled K-major; 1), stride byte offset =
// 1024 B between 8-row atoms, fixed version bits 46-47 = 1, swizzle mode
// SWIZZLE_128B (2) in bits 61-63.  The tile base is 1024-byte aligned.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (encoded)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D fp32 (bits 4-5 = 1), A and B bf16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 16 consecutive fp32 accumulator columns of this thread's row.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Copy rows [r0, r0 + rows) x K-block [k0, k0 + 64) of a K-major bf16 matrix
// into a swizzled tile; rows >= nrows and columns >= ncols read as zero.
__device__ __forceinline__ void load_tile(uint8_t *tile, const __nv_bfloat16 *src, int ld, int r0,
                                          int rows, int nrows, int k0, int ncols)
{
    for (int idx = threadIdx.x; idx < rows * 8; idx += blockDim.x) {
        const int r = idx >> 3, c = idx & 7;
        const int gr = r0 + r, gk = k0 + c * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gr < nrows) {
            const __nv_bfloat16 *p = src + (size_t)gr * ld + gk;
            if (gk + 8 <= ncols && ((reinterpret_cast<uintptr_t>(p) & 15u) == 0)) {
                v = *reinterpret_cast<const uint4 *>(p);
            } else {
                uint32_t w[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint16_t lo = gk + 2 * j < ncols ? __bfloat16_as_ushort(p[2 * j]) : 0;
                    const uint16_t hi = gk + 2 * j + 1 < ncols ? __bfloat16_as_ushort(p[2 * j + 1]) : 0;
                    w[j] = (uint32_t)lo | ((uint32_t)hi << 16);
                }
                v = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        *reinterpret_cast<uint4 *>(tile + r * 128 + ((c ^ (r & 7)) << 4)) = v;
    }
}

template <int N>
__global__ void __launch_bounds__(128, 1) k_gemm_bf16(const GemmArgs g)
{
    // two stages: the tiles of K block i + 1 are written while the MMAs of
    // block i run; a stage is rewritten only after the MMAs that read it
    // completed (its own mbarrier)
    extern __shared__ uint8_t dsmem[];  // gemm_smem_bytes(N): two stages, 1024-byte aligned below
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_tmem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TM;
    // the swizzled tiles start on 1024-byte boundaries (the descriptors' atoms)
    uint8_t *const tiles = dsmem + ((1024u - (smem_u32(dsmem) & 1023u)) & 1023u);
    // stage st: A tile at tiles + st * TM * 128, B tile at tiles + 2 TM 128 + st * N * 128

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    constexpr uint32_t idesc = instr_desc(TM, N);

    // this CTA's K blocks: [kb0, kb1)
    const int kblocks = (g.k + TK - 1) / TK;
    const int kb0 = blockIdx.y * g.kb_per_split;
    const int kb1 = min(kblocks, kb0 + g.kb_per_split);
    const int nkb = kb1 > kb0 ? kb1 - kb0 : 0;
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
        const int st = i & 1, kb = kb0 + i;
        if (i >= 2) {  // the MMAs of block i - 2 read this stage
            const bool done = mbar_wait_bounded(&s_bar[st], (uint32_t)(((i - 2) >> 1) & 1), MMA_LIMIT_NS);
            if (!__syncthreads_and(done)) {
                ok = false;
                break;
            }
        }
        uint8_t *const sa = tiles + st * (TM * 128);
        uint8_t *const sb = tiles + 2 * (TM * 128) + st * (N * 128);
        load_tile(sa, g.a, g.lda, m0, TM, g.m, kb * TK, g.k);
        load_tile(sb, g.b, g.ldb, 0, N, g.n, kb * TK, g.k);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> async reads
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t ad = smem_desc(smem_u32(sa)), bd = smem_desc(smem_u32(sb));
#pragma unroll
            for (int ks = 0; ks < TK / 16; ++ks)  // 16 bf16 = 32 bytes = 2 descriptor units
                mma_bf16(tmem, ad + 2 * ks, bd + 2 * ks, idesc, (i > 0 || ks > 0) ? 1u : 0u);
            mma_commit(&s_bar[st]);
        }
    }
    if (ok && nkb > 0) {  // the last commit covers every earlier MMA of this thread
        const int last = nkb - 1;
        const bool done = mbar_wait_bounded(&s_bar[last & 1], (uint32_t)((last >> 1) & 1), MMA_LIMIT_NS);
        ok = __syncthreads_and(done) != 0;
    }
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(g.err, ERR_STAGE_TIMEOUT);
    } else if (nkb > 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = m0 + warp * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tmem_ld16(taddr + (uint32_t)c0, v);
            if (row < g.m) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = c0 + i;
                    if (col >= g.n) break;
                    float x = v[i];
                    if (g.accumulate) {
                        atomicAdd(g.d32 + (size_t)row * g.ldd + col, x);
                        continue;
                    }
                    if (g.bias) x += g.bias[col];
                    if (g.relu) x = fmaxf(x, 0.0f);
                    if (g.resid) x += g.resid[(size_t)row * g.ldr + col];
                    if (g.d32) g.d32[(size_t)row * g.ldd + col] = x;
                    if (g.d16) g.d16[(size_t)row * g.ldd + col] = __float2bfloat16(x);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(N)
                     : "memory");
    }
}

// Dynamic shared memory of k_gemm_bf16<N>: two stages of the A and B tiles
// plus room to align them to 1024 bytes.
constexpr int gemm_smem_bytes(int n) { return 2 * (TM * 128 + n * 128) + 1024; }

template <int N>
cudaError_t launch_gemm_tile(const GemmArgs &g, dim3 grid, cudaStream_t s)
{
    static bool attr = false;  // per process: the attribute applies to the kernel
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   gemm_smem_bytes(N));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_gemm_bf16<N><<<grid, 128, gemm_smem_bytes(N), s>>>(g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_bf16(const __nv_bfloat16 *a, int lda, const __nv_bfloat16 *b, int ldb,
                             const float *bias, const float *resid, int ldr, float *d32,
                             __nv_bfloat16 *d16, int ldd, int m, int n, int k, int relu,
                             uint32_t *err, cudaStream_t s)
{
    const int kblocks = (k + TK - 1) / TK;
    GemmArgs g{a, b, bias, resid, d32, d16, m, n, k, lda, ldb, ldd, ldr, relu, err, kblocks > 0 ? kblocks : 1, 0};
    const int grid = (m + TM - 1) / TM;
    if (grid == 0) return cudaSuccess;
    return n <= 64 ? launch_gemm_tile<64>(g, dim3(grid), s) : launch_gemm_tile<128>(g, dim3(grid), s);
}

cudaError_t launch_gemm_bf16_splitk(const __nv_bfloat16 *a, int lda, const __nv_bfloat16 *b, int ldb,
                                    float *d32, int ldd, int m, int n, int k, int max_ctas, uint32_t *err,
                                    cudaStream_t s)
{
    const int kblocks = (k + TK - 1) / TK;
    const int gx = (m + TM - 1) / TM;
    if (gx == 0 || kblocks == 0) return cudaSuccess;
    // split K so that the CTAs cover up to max_ctas SMs, at least two K blocks each
    int splits = max_ctas / gx;
    splits = splits < 1 ? 1 : splits;
    if (splits > (kblocks + 1) / 2) splits = (kblocks + 1) / 2;
    const int per = (kblocks + splits - 1) / splits;
    splits = (kblocks + per - 1) / per;
    GemmArgs g{a, b, nullptr, nullptr, d32, nullptr, m, n, k, lda, ldb, ldd, 0, 0, err, per, 1};
    const dim3 grid(gx, splits);
    return n <= 64 ? launch_gemm_tile<64>(g, grid, s) : launch_gemm_tile<128>(g, grid, s);
}

}  // namespace mmas

using namespace mmas;

extern "C" mmas_status mmas_gemm_bf16(const void *d_a, int32_t lda, const void *d_b, int32_t ldb,
                                      const float *d_bias, float *d_out, int32_t ldd, int32_t m,
                                      int32_t n, int32_t k, int32_t relu, void *stream)
{
    if (!d_a || !d_b || !d_out || m < 0 || k < 0 || n < 1 || n > 128 || lda < k || ldb < k ||
        ldd < n) {
        set_thread_error("mmas_gemm_bf16: need non-NULL A, B, out; 1 <= n <= 128; lda, ldb >= k; ldd >= n");
        return MMAS_EINVAL;
    }
    uint32_t *err = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMallocAsync(&err, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess)
        e = launch_gemm_bf16(static_cast<const __nv_bfloat16 *>(d_a), lda,
                             static_cast<const __nv_bfloat16 *>(d_b), ldb, d_bias, nullptr, 0, d_out,
                             nullptr, ldd, m, n, k, relu, err, s);
    uint32_t h_err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (err) cudaFreeAsync(err, s);
    if (e != cudaSuccess) {
        set_thread_error(std::string("mmas_gemm_bf16: ") + cudaGetErrorString(e));
        return MMAS_ECUDA;
    }
    if (h_err) {
        set_thread_error("mmas_gemm_bf16: an MMA did not complete in time");
        return MMAS_ETIMEOUT;
    }
    return MMAS_OK;
}

extern "C" mmas_status mmas_gemm_bf16_acc(const void *d_a, int32_t lda, const void *d_b, int32_t ldb, float *d_out,
                                          int32_t ldd, int32_t m, int32_t n, int32_t k, void *stream)
{
    if (!d_a || !d_b || !d_out || m < 0 || k < 0 || n < 1 || n > 128 || lda < k || ldb < k || ldd < n) {
        set_thread_error("mmas_gemm_bf16_acc: need non-NULL A, B, out; 1 <= n <= 128; lda, ldb >= k; ldd >= n");
        return MMAS_EINVAL;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint32_t *err = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMallocAsync(&err, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess)
        e = launch_gemm_bf16_splitk(static_cast<const __nv_bfloat16 *>(d_a), lda,
                                    static_cast<const __nv_bfloat16 *>(d_b), ldb, d_out, ldd, m, n, k, sms, err, s);
    uint32_t h_err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (err) cudaFreeAsync(err, s);
    if (e != cudaSuccess) {
        set_thread_error(std::string("mmas_gemm_bf16_acc: ") + cudaGetErrorString(e));
        return MMAS_ECUDA;
    }
    if (h_err) {
        set_thread_error("mmas_gemm_bf16_acc: an MMA did not complete in time");
        return MMAS_ETIMEOUT;
    }
    return MMAS_OK;
}
