// Learned edge prior (mmas_prior_*, include/mmas.h): a 3-layer message-passing
// network over each node's 16 nearest neighbours (the first 16 entries of the
// colony's candidate lists) that scores every candidate edge; its edge
// probabilities replace eta^beta in choice_info (an extension of this library;
// the paper's heuristic is eta = 1/d).
//
//   F0   [n][8]   bf16 features (box-centred coordinates, four neighbour
//                 distances / D, a constant), D = max_i d(i, nn[i][15])
//   h0 = relu(F0 W0^T + b0)                                  fp32 + bf16 copy
//   z_l = [h | mean_k h_nn]  (bf16, [n][128])
//   h_l = relu(z_l W_l^T + b_l) + h_{l-1},  l = 1..3          fp32 + bf16 copy
//   q = h3 Wq^T;  s[i][k] = <q_i, h3[nn[i][k]]> / 8 + a dn[i][k] + c
//
// Every dense contraction (the input, layer and query products, and in
// training the weight and input gradients) runs on the tensor cores through
// launch_gemm_bf16 (tcgen05, FP32 accumulation).  The gathers, scatters, score
// dots and the Adam update are small plain kernels.  Training on one colony's
// instance and an elite tour minimises the mean binary cross-entropy of
// sigmoid(s) against y[i][k] = [(i, nn[i][k]) is a tour edge].
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace mmas;

namespace mmas {
cudaError_t launch_gemm_bf16(const __nv_bfloat16 *a, int lda, const __nv_bfloat16 *b, int ldb,
                             const float *bias, const float *resid, int ldr, float *d32,
                             __nv_bfloat16 *d16, int ldd, int m, int n, int k, int relu,
                             uint32_t *err, cudaStream_t s);
cudaError_t launch_gemm_bf16_splitk(const __nv_bfloat16 *a, int lda, const __nv_bfloat16 *b, int ldb,
                                    float *d32, int ldd, int m, int n, int k, int max_ctas, uint32_t *err,
                                    cudaStream_t s);
}

namespace {

constexpr int H = 64, KN = 16, FIN = 8;
// parameter offsets (fp32 vector; layout in include/mmas.h)
constexpr int O_W0 = 0, O_B0 = O_W0 + H * FIN;
constexpr int O_W1 = O_B0 + H, O_B1 = O_W1 + H * 2 * H;
constexpr int O_W2 = O_B1 + H, O_B2 = O_W2 + H * 2 * H;
constexpr int O_W3 = O_B2 + H, O_B3 = O_W3 + H * 2 * H;
constexpr int O_WQ = O_B3 + H, O_A = O_WQ + H * H, O_C = O_A + 1, NPARAM = O_C + 1;
static_assert(NPARAM == MMAS_PRIOR_PARAMS, "parameter layout");
__host__ __device__ constexpr int o_wl(int l) { return l == 1 ? O_W1 : (l == 2 ? O_W2 : O_W3); }
__host__ __device__ constexpr int o_bl(int l) { return l == 1 ? O_B1 : (l == 2 ? O_B2 : O_B3); }

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + __expf(-x)); }

// exact integer extremes of the coordinates and of the 16th-neighbour distance
__global__ void k_prior_extremes(const int2 *xy, const int32_t *dist, const int32_t *nn, int n, int ld,
                                 int cl, int *ext /* minx, maxx, miny, maxy, D */)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int2 p = xy[i];
        atomicMin(ext + 0, p.x);
        atomicMax(ext + 1, p.x);
        atomicMin(ext + 2, p.y);
        atomicMax(ext + 3, p.y);
        atomicMax(ext + 4, dist[(size_t)i * ld + nn[(size_t)i * cl + KN - 1]]);
    }
}

__global__ void k_prior_features(const int2 *xy, const int32_t *dist, const int32_t *cand, int n, int ld,
                                 int cl, const int *ext, bf16 *F, float *dn, int32_t *nn16)
{
    const double cx = ((double)ext[0] + (double)ext[1]) / 2.0, cy = ((double)ext[2] + (double)ext[3]) / 2.0;
    const double s = (double)max(max(ext[1] - ext[0], ext[3] - ext[2]), 1);
    const double D = (double)max(ext[4], 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int2 p = xy[i];
        float dk[KN];
        for (int k = 0; k < KN; ++k) {
            const int j = cand[(size_t)i * cl + k];
            nn16[(size_t)i * KN + k] = j;
            dk[k] = (float)((double)dist[(size_t)i * ld + j] / D);
            dn[(size_t)i * KN + k] = dk[k];
        }
        const float f[FIN] = {(float)(((double)p.x - cx) / s), (float)(((double)p.y - cy) / s), dk[0], dk[1],
                              dk[3], dk[15], 1.0f, 0.0f};
        for (int c = 0; c < FIN; ++c) F[(size_t)i * FIN + c] = __float2bfloat16(f[c]);
    }
}

// z[i] = [hb[i] | bf16(mean_k hb[nn[i][k]])], the mean accumulated in fp32, k in order
__global__ void k_prior_gather(const bf16 *hb, const int32_t *nn, int n, bf16 *z)
{
    const size_t total = (size_t)n * H;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / H), c = (int)(e % H);
        float acc = 0.0f;
        for (int k = 0; k < KN; ++k) acc += __bfloat162float(hb[(size_t)nn[(size_t)i * KN + k] * H + c]);
        z[(size_t)i * 2 * H + c] = hb[e];
        z[(size_t)i * 2 * H + H + c] = __float2bfloat16(acc * (1.0f / KN));
    }
}

// s[i][k] = <q_i, hb[nn[i][k]]> / 8 + a dn + c   (fp32, c in order)
__global__ void k_prior_scores(const float *q, const bf16 *hb, const int32_t *nn, const float *dn,
                               const float *params, int n, float *s)
{
    const float a = params[O_A], c0 = params[O_C];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * KN; e += gridDim.x * blockDim.x) {
        const int i = e / KN;
        const bf16 *hj = hb + (size_t)nn[e] * H;
        const float *qi = q + (size_t)i * H;
        float dot = 0.0f;
        for (int c = 0; c < H; ++c) dot += qi[c] * __bfloat162float(hj[c]);
        s[e] = dot * 0.125f + a * dn[e] + c0;
    }
}

// fp32 parameters -> bf16 weights (row-major [out][in]) and their transposes
__global__ void k_prior_pack(const float *params, bf16 *w0, bf16 *wl, bf16 *wlt, bf16 *wq, bf16 *wqt)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int e = t; e < H * FIN; e += stride) w0[e] = __float2bfloat16(params[O_W0 + e]);
    for (int l = 1; l <= 3; ++l)
        for (int e = t; e < H * 2 * H; e += stride) {
            const int o = e / (2 * H), i = e % (2 * H);
            const bf16 v = __float2bfloat16(params[o_wl(l) + e]);
            wl[(size_t)(l - 1) * H * 2 * H + e] = v;
            wlt[(size_t)(l - 1) * H * 2 * H + (size_t)i * H + o] = v;
        }
    for (int e = t; e < H * H; e += stride) {
        const int o = e / H, i = e % H;
        const bf16 v = __float2bfloat16(params[O_WQ + e]);
        wq[e] = v;
        wqt[(size_t)i * H + o] = v;
    }
}

__global__ void k_prior_succ(const int32_t *tour, int n, int2 *sp)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        sp[tour[t]] = make_int2(tour[t + 1 == n ? 0 : t + 1], tour[t == 0 ? n - 1 : t - 1]);
}

__global__ void k_prior_y(const int2 *sp, const int32_t *nn, int n, float *y)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * KN; e += gridDim.x * blockDim.x) {
        const int2 v = sp[e / KN];
        y[e] = (nn[e] == v.x || nn[e] == v.y) ? 1.0f : 0.0f;
    }
}

// ds = (sigmoid(s) - y) / (n K); loss sum; gradients of a and c; dq; dh3 scatter
__global__ void k_prior_head_back(const float *s, const float *y, const float *dn, const float *q,
                                  const bf16 *hb, const int32_t *nn, int n, float *dq, float *dh,
                                  float *grad, double *loss)
{
    const float inv = 1.0f / ((float)n * KN);
    double lsum = 0.0;
    float ga = 0.0f, gc = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float dqi[H];
        for (int c = 0; c < H; ++c) dqi[c] = 0.0f;
        for (int k = 0; k < KN; ++k) {
            const int e = i * KN + k;
            const float sv = s[e], yv = y[e];
            lsum += (double)fmaxf(sv, 0.0f) - (double)sv * yv + log1p(exp(-fabs((double)sv)));
            const float ds = (sigmoidf_(sv) - yv) * inv;
            ga += ds * dn[e];
            gc += ds;
            const int j = nn[e];
            for (int c = 0; c < H; ++c) {
                dqi[c] += ds * __bfloat162float(hb[(size_t)j * H + c]) * 0.125f;
                atomicAdd(dh + (size_t)j * H + c, ds * q[(size_t)i * H + c] * 0.125f);
            }
        }
        for (int c = 0; c < H; ++c) dq[(size_t)i * H + c] = dqi[c];
    }
    atomicAdd(grad + O_A, ga);
    atomicAdd(grad + O_C, gc);
    atomicAdd(loss, lsum);
}

// da = dh * [h_l - h_{l-1} > 0] (bf16 copy and bf16 transpose for the GEMMs);
// for the input layer (hprev == nullptr) the mask is [h0 > 0]
__global__ void k_prior_relu_back(const float *dh, const float *hl, const float *hprev, int n, bf16 *dab,
                                  bf16 *daT, float *dbias)
{
    const size_t total = (size_t)n * H;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / H), c = (int)(e % H);
        const float r = hprev ? hl[e] - hprev[e] : hl[e];
        const float da = r > 0.0f ? dh[e] : 0.0f;
        dab[e] = __float2bfloat16(da);
        daT[(size_t)c * n + i] = __float2bfloat16(da);
        if (da != 0.0f) atomicAdd(dbias + c, da);
    }
}

// dh_{l-1} = dh + dz[:, :H];  dh_{l-1}[nn[i][k]] += dz[i][H + c] / K
__global__ void k_prior_layer_back(const float *dh, const float *dz, const int32_t *nn, int n, float *dhp)
{
    const size_t total = (size_t)n * H;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / H), c = (int)(e % H);
        atomicAdd(dhp + e, dh[e] + dz[(size_t)i * 2 * H + c]);
        const float g = dz[(size_t)i * 2 * H + H + c] * (1.0f / KN);
        for (int k = 0; k < KN; ++k) atomicAdd(dhp + (size_t)nn[(size_t)i * KN + k] * H + c, g);
    }
}

// x [rows][cols] bf16 -> xT [cols][rows]
__global__ void k_transpose_bf16(const bf16 *x, int rows, int cols, int ldx, bf16 *xT)
{
    __shared__ bf16 tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy, c = c0 + threadIdx.x;
        tile[dy][threadIdx.x] = (r < rows && c < cols) ? x[(size_t)r * ldx + c] : __float2bfloat16(0.0f);
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int c = c0 + dy, r = r0 + threadIdx.x;
        if (c < cols && r < rows) xT[(size_t)c * rows + r] = tile[threadIdx.x][dy];
    }
}

// x [n][H] fp32 -> bf16 row-major and transposed [H][n]
__global__ void k_prior_cvt(const float *x, int n, bf16 *xb, bf16 *xT)
{
    const size_t total = (size_t)n * H;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const bf16 v = __float2bfloat16(x[e]);
        xb[e] = v;
        xT[(size_t)(e % H) * n + e / H] = v;
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int count, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const float gv = g[e];
        const float mv = b1 * m[e] + (1.0f - b1) * gv, vv = b2 * v[e] + (1.0f - b2) * gv * gv;
        m[e] = mv;
        v[e] = vv;
        p[e] -= lr * (mv / c1) / (sqrtf(vv / c2) + eps);
    }
}

// eta^beta' of row i: the 16 candidates take sigmoid(s); every other node j
// keeps the distance heuristic rescaled so that the farthest candidate's value
// maps to the row's smallest candidate probability
__global__ void k_prior_apply(const float *s, const int32_t *nn, int n, int ld, float *eb)
{
    __shared__ float s_scale;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        float *row = eb + (size_t)i * ld;
        if (threadIdx.x == 0) {
            float pmin = 1.0f;
            for (int k = 0; k < KN; ++k) pmin = fminf(pmin, sigmoidf_(s[i * KN + k]));
            const float far = row[nn[i * KN + KN - 1]];
            s_scale = far > 0.0f ? pmin / far : 0.0f;
        }
        __syncthreads();
        const float sc = s_scale;
        for (int j = threadIdx.x; j < n; j += blockDim.x) row[j] *= sc;
        __syncthreads();
        if (threadIdx.x < KN) row[nn[i * KN + threadIdx.x]] = sigmoidf_(s[i * KN + threadIdx.x]);
        __syncthreads();
    }
}

// eta^beta <- eta^beta sigmoid(s)^gamma on each row's candidate edges and
// eta^beta (min_k sigmoid(s_ik))^gamma elsewhere (the distance order among
// the other entries is kept).
__global__ void k_prior_weight(const float *s, const int32_t *nn, int n, int ld, float gamma, float *eb)
{
    __shared__ float s_scale;
    __shared__ float s_cand[KN];
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        float *row = eb + (size_t)i * ld;
        if (threadIdx.x == 0) {
            float pmin = 1.0f;
            for (int k = 0; k < KN; ++k) pmin = fminf(pmin, sigmoidf_(s[i * KN + k]));
            s_scale = powf(pmin, gamma);
        }
        if (threadIdx.x < KN)
            s_cand[threadIdx.x] = row[nn[i * KN + threadIdx.x]] * powf(sigmoidf_(s[i * KN + threadIdx.x]), gamma);
        __syncthreads();
        const float sc = s_scale;
        for (int j = threadIdx.x; j < n; j += blockDim.x) row[j] *= sc;
        __syncthreads();
        if (threadIdx.x < KN) row[nn[i * KN + threadIdx.x]] = s_cand[threadIdx.x];
        __syncthreads();
    }
}

}  // namespace

struct mmas_prior {
    int device = 0;
    float *params = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    bf16 *w0 = nullptr, *wl = nullptr, *wlt = nullptr, *wq = nullptr, *wqt = nullptr;
    int adam_t = 0;
    int num_sms = 0;  // of the prior's device, looked up at the first split-K product
    bool packed = false;
    // workspace for an n-node instance
    int cap = 0;
    int *ext = nullptr;
    bf16 *F = nullptr, *FT = nullptr, *hb[4] = {}, *z[4] = {}, *zT = nullptr, *dab = nullptr, *daT = nullptr,
         *hbT = nullptr, *dqb = nullptr, *dqT = nullptr;
    float *dn = nullptr, *h[4] = {}, *q = nullptr, *s = nullptr, *y = nullptr, *dh = nullptr, *dhp = nullptr,
          *dz = nullptr, *dq = nullptr;
    int32_t *nn = nullptr, *tour = nullptr;
    int2 *sp = nullptr;
    double *loss = nullptr;
    uint32_t *err = nullptr;
    std::string errmsg;
};

namespace {

thread_local std::string tl_prior_error;

mmas_status pfail(mmas_prior *p, mmas_status st, const std::string &msg)
{
    if (p)
        p->errmsg = msg;
    else
        tl_prior_error = msg;
    return st;
}

#define PCK(p, call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return pfail((p), e_ == cudaErrorMemoryAllocation ? MMAS_ENOMEM : MMAS_ECUDA,   \
                         std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

void free_work(mmas_prior *p)
{
    void *bufs[] = {p->ext, p->F, p->FT, p->zT, p->dab, p->daT, p->hbT, p->dqb, p->dqT, p->dn, p->q, p->s,
                    p->y, p->dh, p->dhp, p->dz, p->dq, p->nn, p->tour, p->sp};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (int l = 0; l < 4; ++l) {
        if (p->hb[l]) cudaFree(p->hb[l]);
        if (p->z[l]) cudaFree(p->z[l]);
        if (p->h[l]) cudaFree(p->h[l]);
        p->hb[l] = nullptr;
        p->z[l] = nullptr;
        p->h[l] = nullptr;
    }
    p->ext = nullptr; p->F = p->FT = p->zT = p->dab = p->daT = p->hbT = p->dqb = p->dqT = nullptr;
    p->dn = p->q = p->s = p->y = p->dh = p->dhp = p->dz = p->dq = nullptr;
    p->nn = p->tour = nullptr;
    p->sp = nullptr;
    p->cap = 0;
}

mmas_status ensure(mmas_prior *p, int n)
{
    if (n <= p->cap) return MMAS_OK;
    free_work(p);
    const size_t N = (size_t)n;
    PCK(p, device_malloc(&p->ext, 8 * sizeof(int)));
    PCK(p, device_malloc(&p->F, N * FIN * sizeof(bf16)));
    PCK(p, device_malloc(&p->FT, N * FIN * sizeof(bf16)));
    for (int l = 0; l < 4; ++l) {
        PCK(p, device_malloc(&p->hb[l], N * H * sizeof(bf16)));
        PCK(p, device_malloc(&p->h[l], N * H * sizeof(float)));
        PCK(p, device_malloc(&p->z[l], N * 2 * H * sizeof(bf16)));
    }
    PCK(p, device_malloc(&p->zT, N * 2 * H * sizeof(bf16)));
    PCK(p, device_malloc(&p->dab, N * H * sizeof(bf16)));
    PCK(p, device_malloc(&p->daT, N * H * sizeof(bf16)));
    PCK(p, device_malloc(&p->hbT, N * H * sizeof(bf16)));
    PCK(p, device_malloc(&p->dqb, N * H * sizeof(bf16)));
    PCK(p, device_malloc(&p->dqT, N * H * sizeof(bf16)));
    PCK(p, device_malloc(&p->dn, N * KN * sizeof(float)));
    PCK(p, device_malloc(&p->q, N * H * sizeof(float)));
    PCK(p, device_malloc(&p->s, N * KN * sizeof(float)));
    PCK(p, device_malloc(&p->y, N * KN * sizeof(float)));
    PCK(p, device_malloc(&p->dh, N * H * sizeof(float)));
    PCK(p, device_malloc(&p->dhp, N * H * sizeof(float)));
    PCK(p, device_malloc(&p->dz, N * 2 * H * sizeof(float)));
    PCK(p, device_malloc(&p->dq, N * H * sizeof(float)));
    PCK(p, device_malloc(&p->nn, N * KN * sizeof(int32_t)));
    PCK(p, device_malloc(&p->tour, N * sizeof(int32_t)));
    PCK(p, device_malloc(&p->sp, N * sizeof(int2)));
    p->cap = n;
    return MMAS_OK;
}

mmas_status check_colony_for_prior(mmas_prior *p, const mmas_handle *h)
{
    if (!h) return pfail(p, MMAS_EINVAL, "colony handle is NULL");
    if (!h->xy) return pfail(p, MMAS_EINVAL, "the prior needs an instance with coordinates");
    if (h->cl < KN) return pfail(p, MMAS_EINVAL, "the prior needs candidate lists of length >= 16");
    return MMAS_OK;
}

int blocks_for(size_t work, int threads = 256)
{
    const size_t b = (work + threads - 1) / threads;
    return (int)std::min<size_t>(std::max<size_t>(b, 1), 4096);
}

mmas_status gemm(mmas_prior *p, const bf16 *a, int lda, const bf16 *b, int ldb, const float *bias,
                 const float *resid, int ldr, float *d32, bf16 *d16, int ldd, int m, int nn, int k, int relu,
                 cudaStream_t s)
{
    PCK(p, launch_gemm_bf16(a, lda, b, ldb, bias, resid, ldr, d32, d16, ldd, m, nn, k, relu, p->err, s));
    return MMAS_OK;
}

// A weight gradient d32 += A B^T with K = n: K is split over CTAs that add
// their partial products into d32, which the training step zeroed.
mmas_status gemm_wgrad(mmas_prior *p, const bf16 *a, int lda, const bf16 *b, int ldb, float *d32, int ldd, int m,
                       int nn, int k, cudaStream_t s)
{
    if (!p->num_sms) PCK(p, cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    PCK(p, launch_gemm_bf16_splitk(a, lda, b, ldb, d32, ldd, m, nn, k, p->num_sms, p->err, s));
    return MMAS_OK;
}

// Forward pass on colony h's instance; leaves activations and scores in p.
mmas_status forward(mmas_prior *p, mmas_handle *h)
{
    const int n = h->n;
    cudaStream_t s = h->stream;
    mmas_status st = ensure(p, n);
    if (st != MMAS_OK) return st;
    if (!p->packed) {
        k_prior_pack<<<64, 256, 0, s>>>(p->params, p->w0, p->wl, p->wlt, p->wq, p->wqt);
        PCK(p, cudaGetLastError());
        p->packed = true;
    }
    const int init[8] = {INT_MAX, INT_MIN, INT_MAX, INT_MIN, 0, 0, 0, 0};
    PCK(p, cudaMemcpyAsync(p->ext, init, sizeof(init), cudaMemcpyHostToDevice, s));
    k_prior_extremes<<<blocks_for(n), 256, 0, s>>>(h->xy, h->dist, h->cand32, n, h->ld, h->cl, p->ext);
    k_prior_features<<<blocks_for(n), 256, 0, s>>>(h->xy, h->dist, h->cand32, n, h->ld, h->cl, p->ext, p->F,
                                                   p->dn, p->nn);
    PCK(p, cudaGetLastError());
    if ((st = gemm(p, p->F, FIN, p->w0, FIN, p->params + O_B0, nullptr, 0, p->h[0], p->hb[0], H, n, H, FIN, 1, s)))
        return st;
    for (int l = 1; l <= 3; ++l) {
        k_prior_gather<<<blocks_for((size_t)n * H), 256, 0, s>>>(p->hb[l - 1], p->nn, n, p->z[l]);
        PCK(p, cudaGetLastError());
        if ((st = gemm(p, p->z[l], 2 * H, p->wl + (size_t)(l - 1) * H * 2 * H, 2 * H, p->params + o_bl(l),
                       p->h[l - 1], H, p->h[l], p->hb[l], H, n, H, 2 * H, 1, s)))
            return st;
    }
    if ((st = gemm(p, p->hb[3], H, p->wq, H, nullptr, nullptr, 0, p->q, nullptr, H, n, H, H, 0, s))) return st;
    k_prior_scores<<<blocks_for((size_t)n * KN), 256, 0, s>>>(p->q, p->hb[3], p->nn, p->dn, p->params, n, p->s);
    PCK(p, cudaGetLastError());
    return MMAS_OK;
}

mmas_status check_err(mmas_prior *p, cudaStream_t s)
{
    uint32_t e = 0;
    PCK(p, cudaMemcpyAsync(&e, p->err, sizeof(e), cudaMemcpyDeviceToHost, s));
    PCK(p, cudaStreamSynchronize(s));
    if (e) return pfail(p, MMAS_ETIMEOUT, "a tensor-core product did not complete in time");
    return MMAS_OK;
}

}  // namespace

extern "C" {

mmas_status mmas_prior_create(const float *params, int32_t device, mmas_prior **out)
{
    if (!out) return pfail(nullptr, MMAS_EINVAL, "out must be non-NULL");
    *out = nullptr;
    mmas_prior *p = new (std::nothrow) mmas_prior();
    if (!p) return pfail(nullptr, MMAS_ENOMEM, "host allocation failed");
    p->device = device;
    int prev = -1;
    cudaGetDevice(&prev);
    auto fail_all = [&](mmas_status st) {
        tl_prior_error = p->errmsg;
        mmas_prior_destroy(p);
        if (prev >= 0) cudaSetDevice(prev);
        return st;
    };
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        p->errmsg = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return fail_all(MMAS_ECUDA);
    }
    const size_t pb = NPARAM * sizeof(float);
    void **fb[] = {(void **)&p->params, (void **)&p->grad, (void **)&p->adam_m, (void **)&p->adam_v};
    for (void **b : fb) {
        if ((e = device_malloc(b, pb)) != cudaSuccess || (e = cudaMemset(*b, 0, pb)) != cudaSuccess) {
            p->errmsg = std::string("cudaMalloc: ") + cudaGetErrorString(e);
            return fail_all(MMAS_ENOMEM);
        }
    }
    const size_t wsz[5] = {H * FIN, 3 * H * 2 * H, 3 * H * 2 * H, H * H, H * H};
    bf16 **wb[5] = {&p->w0, &p->wl, &p->wlt, &p->wq, &p->wqt};
    for (int i = 0; i < 5; ++i)
        if ((e = device_malloc(wb[i], wsz[i] * sizeof(bf16))) != cudaSuccess) {
            p->errmsg = std::string("cudaMalloc: ") + cudaGetErrorString(e);
            return fail_all(MMAS_ENOMEM);
        }
    if ((e = device_malloc(&p->err, sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemset(p->err, 0, sizeof(uint32_t))) != cudaSuccess ||
        (e = device_malloc(&p->loss, sizeof(double))) != cudaSuccess) {
        p->errmsg = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return fail_all(MMAS_ENOMEM);
    }
    if (params && (e = cudaMemcpy(p->params, params, pb, cudaMemcpyHostToDevice)) != cudaSuccess) {
        p->errmsg = std::string("cudaMemcpy: ") + cudaGetErrorString(e);
        return fail_all(MMAS_ECUDA);
    }
    if (prev >= 0) cudaSetDevice(prev);
    *out = p;
    return MMAS_OK;
}

mmas_status mmas_prior_set_params(mmas_prior *p, const float *params)
{
    if (!p || !params) return pfail(p, MMAS_EINVAL, "prior and params must be non-NULL");
    PCK(p, cudaMemcpy(p->params, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    p->packed = false;
    p->adam_t = 0;
    PCK(p, cudaMemset(p->adam_m, 0, NPARAM * sizeof(float)));
    PCK(p, cudaMemset(p->adam_v, 0, NPARAM * sizeof(float)));
    return MMAS_OK;
}

mmas_status mmas_prior_get_params(mmas_prior *p, float *params)
{
    if (!p || !params) return pfail(p, MMAS_EINVAL, "prior and params must be non-NULL");
    PCK(p, cudaDeviceSynchronize());
    PCK(p, cudaMemcpy(params, p->params, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return MMAS_OK;
}

mmas_status mmas_prior_get_state(mmas_prior *p, float *m, float *v, float *grad, int32_t *step)
{
    if (!p) return pfail(nullptr, MMAS_EINVAL, "prior is NULL");
    PCK(p, cudaDeviceSynchronize());
    if (m) PCK(p, cudaMemcpy(m, p->adam_m, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    if (v) PCK(p, cudaMemcpy(v, p->adam_v, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    if (grad) PCK(p, cudaMemcpy(grad, p->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    if (step) *step = p->adam_t;
    return MMAS_OK;
}

mmas_status mmas_prior_set_state(mmas_prior *p, const float *m, const float *v, int32_t step)
{
    if (!p || !m || !v) return pfail(p, MMAS_EINVAL, "prior, m and v must be non-NULL");
    if (step < 0) return pfail(p, MMAS_EINVAL, "step must be >= 0");
    for (int i = 0; i < NPARAM; ++i)
        if (!(v[i] >= 0.0f) || !std::isfinite(v[i]) || !std::isfinite(m[i]))
            return pfail(p, MMAS_EINVAL, "m must be finite and v finite and >= 0");
    PCK(p, cudaDeviceSynchronize());
    PCK(p, cudaMemcpy(p->adam_m, m, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    PCK(p, cudaMemcpy(p->adam_v, v, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    p->adam_t = step;
    return MMAS_OK;
}

mmas_status mmas_prior_scores(mmas_prior *p, mmas_handle *h, float *scores)
{
    if (!p || !scores) return pfail(p, MMAS_EINVAL, "prior and scores must be non-NULL");
    mmas_status st = check_colony_for_prior(p, h);
    if (st != MMAS_OK) return st;
    if ((st = forward(p, h)) != MMAS_OK) return st;
    PCK(p, cudaMemcpyAsync(scores, p->s, (size_t)h->n * KN * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    return check_err(p, h->stream);
}

mmas_status mmas_prior_train(mmas_prior *p, mmas_handle *h, const int32_t *tour, int32_t steps, float lr,
                             float *loss_out)
{
    if (!p || !tour || steps < 1 || !(lr > 0.0f))
        return pfail(p, MMAS_EINVAL, "need a prior, a tour, steps >= 1 and lr > 0");
    mmas_status st = check_colony_for_prior(p, h);
    if (st != MMAS_OK) return st;
    const int n = h->n;
    {
        std::vector<char> seen(n, 0);
        for (int i = 0; i < n; ++i) {
            if (tour[i] < 0 || tour[i] >= n || seen[tour[i]])
                return pfail(p, MMAS_EINVAL, "tour must be a permutation of 0..n-1");
            seen[tour[i]] = 1;
        }
    }
    if ((st = ensure(p, n)) != MMAS_OK) return st;
    cudaStream_t s = h->stream;
    PCK(p, cudaMemcpyAsync(p->tour, tour, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_prior_succ<<<blocks_for(n), 256, 0, s>>>(p->tour, n, p->sp);
    auto transpose = [&](const bf16 *x, int rows, int cols, bf16 *xT) {
        dim3 tb(32, 8), tg((cols + 31) / 32, (rows + 31) / 32);
        k_transpose_bf16<<<tg, tb, 0, s>>>(x, rows, cols, cols, xT);
    };
    for (int it = 0; it < steps; ++it) {
        if ((st = forward(p, h)) != MMAS_OK) return st;
        if (it == 0) k_prior_y<<<blocks_for((size_t)n * KN), 256, 0, s>>>(p->sp, p->nn, n, p->y);
        PCK(p, cudaMemsetAsync(p->grad, 0, NPARAM * sizeof(float), s));
        PCK(p, cudaMemsetAsync(p->dh, 0, (size_t)n * H * sizeof(float), s));
        PCK(p, cudaMemsetAsync(p->loss, 0, sizeof(double), s));
        // scores: loss, d(a), d(c), dq, and dh3 from the neighbour side of each dot
        k_prior_head_back<<<blocks_for(n, 128), 128, 0, s>>>(p->s, p->y, p->dn, p->q, p->hb[3], p->nn, n, p->dq,
                                                             p->dh, p->grad, p->loss);
        k_prior_cvt<<<blocks_for((size_t)n * H), 256, 0, s>>>(p->dq, n, p->dqb, p->dqT);
        transpose(p->hb[3], n, H, p->hbT);
        PCK(p, cudaGetLastError());
        // dWq = dq^T h3 ;  dh3 += dq Wq
        if ((st = gemm_wgrad(p, p->dqT, n, p->hbT, n, p->grad + O_WQ, H, H, H, n, s))) return st;
        if ((st = gemm(p, p->dqb, H, p->wqt, H, nullptr, p->dh, H, p->dh, nullptr, H, n, H, H, 0, s))) return st;
        for (int l = 3; l >= 1; --l) {
            // da = dh on the active units; db_l; dW_l = da^T z_l; dz = da W_l
            k_prior_relu_back<<<blocks_for((size_t)n * H), 256, 0, s>>>(p->dh, p->h[l], p->h[l - 1], n, p->dab,
                                                                       p->daT, p->grad + o_bl(l));
            transpose(p->z[l], n, 2 * H, p->zT);
            PCK(p, cudaGetLastError());
            if ((st = gemm_wgrad(p, p->daT, n, p->zT, n, p->grad + o_wl(l), 2 * H, H, 2 * H, n, s))) return st;
            if ((st = gemm(p, p->dab, H, p->wlt + (size_t)(l - 1) * H * 2 * H, H, nullptr, nullptr, 0, p->dz, nullptr,
                           2 * H, n, 2 * H, H, 0, s)))
                return st;
            // dh_{l-1} = dh + dz[:, :H] + the neighbour-mean part scattered back
            PCK(p, cudaMemsetAsync(p->dhp, 0, (size_t)n * H * sizeof(float), s));
            k_prior_layer_back<<<blocks_for((size_t)n * H), 256, 0, s>>>(p->dh, p->dz, p->nn, n, p->dhp);
            PCK(p, cudaGetLastError());
            std::swap(p->dh, p->dhp);
        }
        // input layer: da0 = dh on h0 > 0;  dW0 = da0^T F0;  db0
        k_prior_relu_back<<<blocks_for((size_t)n * H), 256, 0, s>>>(p->dh, p->h[0], nullptr, n, p->dab, p->daT,
                                                                   p->grad + O_B0);
        transpose(p->F, n, FIN, p->FT);
        PCK(p, cudaGetLastError());
        if ((st = gemm_wgrad(p, p->daT, n, p->FT, n, p->grad + O_W0, FIN, H, FIN, n, s))) return st;
        // Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected)
        p->adam_t += 1;
        // bias corrections 1 - beta^t of the single-precision betas, in double
        // (1 - beta2^t loses most of a float's digits to cancellation), rounded once
        const float c1 = (float)(1.0 - pow((double)0.9f, (double)p->adam_t));
        const float c2 = (float)(1.0 - pow((double)0.999f, (double)p->adam_t));
        k_adam<<<blocks_for(NPARAM), 256, 0, s>>>(p->params, p->grad, p->adam_m, p->adam_v, NPARAM, lr, 0.9f, 0.999f,
                                                  1e-8f, c1, c2);
        PCK(p, cudaGetLastError());
        p->packed = false;
    }
    double lsum = 0.0;
    PCK(p, cudaMemcpyAsync(&lsum, p->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    if ((st = check_err(p, s)) != MMAS_OK) return st;
    if (loss_out) *loss_out = (float)(lsum / ((double)n * KN));
    return MMAS_OK;
}

mmas_status mmas_prior_grad(mmas_prior *p, mmas_handle *h, const int32_t *tour, float *grad_out, float *loss_out)
{
    if (!p || !grad_out) return pfail(p, MMAS_EINVAL, "prior and grad_out must be non-NULL");
    // one training step at lr = 0 would still move Adam's moments; instead run
    // the step's gradient pass and restore the parameters and moments
    std::vector<float> keep(NPARAM), km(NPARAM), kv(NPARAM);
    PCK(p, cudaDeviceSynchronize());
    PCK(p, cudaMemcpy(keep.data(), p->params, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    PCK(p, cudaMemcpy(km.data(), p->adam_m, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    PCK(p, cudaMemcpy(kv.data(), p->adam_v, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    const int t = p->adam_t;
    mmas_status st = mmas_prior_train(p, h, tour, 1, 1e-30f, loss_out);
    if (st != MMAS_OK) return st;
    PCK(p, cudaMemcpy(grad_out, p->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    PCK(p, cudaMemcpy(p->params, keep.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    PCK(p, cudaMemcpy(p->adam_m, km.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    PCK(p, cudaMemcpy(p->adam_v, kv.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    p->adam_t = t;
    p->packed = false;
    return MMAS_OK;
}

mmas_status mmas_prior_apply(mmas_prior *p, mmas_handle *h)
{
    if (!p) return pfail(nullptr, MMAS_EINVAL, "prior is NULL");
    mmas_status st = check_colony_for_prior(p, h);
    if (st != MMAS_OK) return st;
    if ((st = forward(p, h)) != MMAS_OK) return st;
    cudaStream_t s = h->stream;
    PCK(p, launch_eta_beta(h->dist, h->n, h->ld, (double)h->p.beta, h->eb, h->ebt, h->maxd_val, s));
    k_prior_apply<<<std::min(h->n, 4096), 256, 0, s>>>(p->s, p->nn, h->n, h->ld, h->eb);
    PCK(p, cudaGetLastError());
    UpdateArgs refresh = h->uargs;
    refresh.evaporate = 0;
    refresh.nbr = nullptr;
    PCK(p, launch_update(refresh, h->num_sms, s));
    return check_err(p, s);
}

mmas_status mmas_prior_apply_weighted(mmas_prior *p, mmas_handle *h, float gamma)
{
    if (!p) return pfail(nullptr, MMAS_EINVAL, "prior is NULL");
    if (!(gamma >= 0.0f) || gamma > 64.0f) return pfail(p, MMAS_EINVAL, "gamma must be in [0, 64]");
    mmas_status st = check_colony_for_prior(p, h);
    if (st != MMAS_OK) return st;
    if ((st = forward(p, h)) != MMAS_OK) return st;
    cudaStream_t s = h->stream;
    PCK(p, launch_eta_beta(h->dist, h->n, h->ld, (double)h->p.beta, h->eb, h->ebt, h->maxd_val, s));
    k_prior_weight<<<std::min(h->n, 4096), 256, 0, s>>>(p->s, p->nn, h->n, h->ld, gamma, h->eb);
    PCK(p, cudaGetLastError());
    UpdateArgs refresh = h->uargs;
    refresh.evaporate = 0;
    refresh.nbr = nullptr;
    PCK(p, launch_update(refresh, h->num_sms, s));
    return check_err(p, s);
}

void mmas_prior_destroy(mmas_prior *p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    free_work(p);
    void *bufs[] = {p->params, p->grad, p->adam_m, p->adam_v, p->w0, p->wl, p->wlt, p->wq, p->wqt, p->err, p->loss};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete p;
}

const char *mmas_prior_last_error(const mmas_prior *p) { return p ? p->errmsg.c_str() : tl_prior_error.c_str(); }

}  // extern "C"
