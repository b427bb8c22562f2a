// Learned surrogate of the per-mode kernel table g^k(d) for far pairs.
//
// A multilayer perceptron 4 -> H -> H -> H -> 6 with SiLU activations maps the
// features of a (difference d, wavenumber k >= 1) pair,
//     x = (q r / 32, d_x / r, d_y / r, ln(r) / 5),   r = |d|,  q = 2 pi k / (L c),
// to the six independent reals of g^k(d) (Re g11, Re g12, Re g22, Re g33,
// Im g13, Im g23) divided by the smooth decay factor
//     s(q, r) = exp(-q r) / (c sqrt(1 + q r)),
// so that the targets are O(1) although the modes decay exponentially in q r.
// It is trained on the plan's own exact FP64 table (the tables the method
// itself generates) by the kernels of this file: a tiled FP32 GEMM used for
// the forward pass and both backward products, SiLU and its derivative, the
// mean-squared loss, bias reductions and Adam.  For inference the weights are
// rounded to bf16 values and the products accumulate in FP32.
//
// Use in the pad update: a plan in a CUDA-core FP32 or tensor-core precision
// can stream its table one mode at a time: for each k >= 1 a slice
// [Dy][Dx][6] is assembled from the exact table for |d| < r_min (near field)
// and from the network for |d| >= r_min, and the contraction of that mode
// reads the slice, so only one slice (not K of them) is resident.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <random>
#include <vector>

#include "fbc_internal.cuh"

struct fbc_surrogate {
    int width = 128;
    int n_params = 0;
    int off[8];          // W1 b1 W2 b2 W3 b3 W4 b4
    float* d_p = nullptr;      // parameters (FP32 master)
    float* d_pb = nullptr;     // parameters rounded to bf16 values (inference)
    float* d_g = nullptr;      // gradients
    float* d_m = nullptr;      // Adam first moment
    float* d_v = nullptr;      // Adam second moment
    int step = 0;
    // training scratch (sized for the largest batch used)
    int cap = 0;
    float* d_act = nullptr;    // Z1 A1 Z2 A2 Z3 A3 (cap x H each), Y, dY (cap x 6), T, B0, B1 (cap x H)
    double* d_loss = nullptr;
};

namespace fbc {

// Beyond q r = kQrCut an entry of mode k >= 1 is below exp(-16) ~ 1e-7 of its
// value at q r -> 0 and, after the roundoff the Richardson weights amplify,
// no longer carries a trustworthy FP64 value: the surrogate serves it as zero
// and is trained only below the cut.
constexpr double kQrCut = 16.0;
namespace {

constexpr int kOut = 6;

// ---- generic FP32 GEMM: C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias) (+ beta C) ----
// TA: A stored K x M (transposed); TB: B stored N x K (transposed).
template <bool TA, bool TB>
__global__ void k_gemm(int M, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
                       float* __restrict__ C, int ldc, const float* __restrict__ bias, float beta) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ float sa[BK][BM + 1];
    __shared__ float sb[BK][BN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 4 x 4 outputs each
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            const int kk = e / BM, mm = e % BM;
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.f;
            if (m < M && k < K) v = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
            sa[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < BN * BK; e += 256) {
            const int kk = e / BN, nn = e % BN;
            const int n = n0 + nn, k = k0 + kk;
            float v = 0.f;
            if (n < N && k < K) v = TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
            sb[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = sa[kk][ty * 4 + i], b[i] = sb[kk][tx * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                float v = acc[i][j];
                if (bias) v += bias[n];
                if (beta != 0.f) v += beta * C[(size_t)m * ldc + n];
                C[(size_t)m * ldc + n] = v;
            }
        }
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    const float s = 1.f / (1.f + expf(-z));
    return s * (1.f + z * (1.f - s));
}

__global__ void k_silu(const float* __restrict__ z, float* __restrict__ a, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        a[i] = silu(z[i]);
}
__global__ void k_silu_back(const float* __restrict__ z, const float* __restrict__ da, float* __restrict__ dz, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dz[i] = da[i] * silu_grad(z[i]);
}
// dY = 2 (Y - T) / (B * 6), loss partials in FP64 (one slot per block, fixed order later)
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy, int n,
                      double* __restrict__ part) {
    __shared__ double red[256];
    double s = 0.0;
    const float sc = 2.f / (float)n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        if (dy) dy[i] = sc * d;
        s += (double)d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
// column sums: db[j] = sum_i dZ[i][j]
__global__ void k_colsum(const float* __restrict__ dz, int rows, int cols, float* __restrict__ db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int i = 0; i < rows; i++) s += dz[(size_t)i * cols + j];
    db[j] = s;
}
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float c1, float c2, float eps) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi, v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}
__global__ void k_round_bf16(const float* __restrict__ p, float* __restrict__ pb, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        pb[i] = __bfloat162float(__float2bfloat16_rn(p[i]));
}

// Features and normalised exact targets of sampled (used difference, k) pairs.
__global__ void k_samples(const int2* __restrict__ used, const int* __restrict__ s_d, const int* __restrict__ s_k,
                          int n, const double* __restrict__ table, int Dx, int Dy, int box_x0, int box_y0, int L,
                          double c, float* __restrict__ X, float* __restrict__ T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 d = used[s_d[i]];
    const int k = s_k[i];
    const double r = sqrt((double)d.x * d.x + (double)d.y * d.y);
    const double q = 2.0 * M_PI * k / (L * c);
    const double qr = q * r;
    X[i * 4 + 0] = (float)(qr / 32.0);
    X[i * 4 + 1] = (float)(d.x / r);
    X[i * 4 + 2] = (float)(d.y / r);
    X[i * 4 + 3] = (float)(log(r) / 5.0);
    if (T) {
        const double inv_s = c * sqrt(1.0 + qr) * exp(qr);
        const double* src = table + (((size_t)k * Dy + (d.y - box_y0)) * Dx + (d.x - box_x0)) * 6;
        for (int j = 0; j < 6; j++) T[i * 6 + j] = (float)(src[j] * inv_s);
    }
}

// Features of every far difference (|d| >= r_min) at one k, for a streamed slice.
__global__ void k_slice_features(const int2* __restrict__ far, int n, int k, int L, double c, float* __restrict__ X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 d = far[i];
    const double r = sqrt((double)d.x * d.x + (double)d.y * d.y);
    const double qr = 2.0 * M_PI * k / (L * c) * r;
    X[i * 4 + 0] = (float)(qr / 32.0);
    X[i * 4 + 1] = (float)(d.x / r);
    X[i * 4 + 2] = (float)(d.y / r);
    X[i * 4 + 3] = (float)(log(r) / 5.0);
}

// Slice assembly: far entries from the network output (times the decay
// factor), near entries copied from the exact FP32 table.
__global__ void k_slice_far(const int2* __restrict__ far, int n, int k, int L, double c, const float* __restrict__ Y,
                            float* __restrict__ slice, int Dx, int box_x0, int box_y0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 d = far[i];
    const double r = sqrt((double)d.x * d.x + (double)d.y * d.y);
    const double qr = 2.0 * M_PI * k / (L * c) * r;
    const double s = qr > kQrCut ? 0.0 : exp(-qr) / (c * sqrt(1.0 + qr));
    float* o = slice + ((size_t)(d.y - box_y0) * Dx + (d.x - box_x0)) * 6;
    for (int j = 0; j < 6; j++) o[j] = (float)(Y[i * 6 + j] * s);
}
__global__ void k_slice_near(const int2* __restrict__ near, int n, int k, const float* __restrict__ near32, int Dx,
                             int box_x0, int box_y0, float* __restrict__ slice) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 d = near[i];
    const size_t cell = (size_t)(d.y - box_y0) * Dx + (d.x - box_x0);
    const float* src = near32 + ((size_t)k * n + i) * 6;
    float* o = slice + cell * 6;
    for (int j = 0; j < 6; j++) o[j] = src[j];
}
// compact exact near-field table: near32[k][i] = FP32 of table[k][near[i]]
__global__ void k_near_gather(const int2* __restrict__ near, int n, int K, const double* __restrict__ table, int Dx,
                              int Dy, int box_x0, int box_y0, float* __restrict__ near32) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)n * K) return;
    const int k = (int)(t / n), i = (int)(t % n);
    const int2 d = near[i];
    const double* src = table + (((size_t)k * Dy + (d.y - box_y0)) * Dx + (d.x - box_x0)) * 6;
    for (int j = 0; j < 6; j++) near32[t * 6 + j] = (float)src[j];
}

int grid_for(size_t n, int bs = 256) { return (int)std::min<size_t>((n + bs - 1) / bs, 152 * 8); }

}  // namespace

// Forward pass of n samples X [n][4] -> Y [n][6]; keeps Z and A of each hidden
// layer in act (layout Z1 A1 Z2 A2 Z3 A3, each cap x H) when `keep`.
cudaError_t surrogate_forward(const fbc_surrogate* S, const float* params, const float* X, int n, float* Y, float* act,
                              int cap, cudaStream_t st) {
    const int H = S->width;
    const float* W[4] = {params + S->off[0], params + S->off[2], params + S->off[4], params + S->off[6]};
    const float* b[4] = {params + S->off[1], params + S->off[3], params + S->off[5], params + S->off[7]};
    const int din[4] = {4, H, H, H}, dout[4] = {H, H, H, kOut};
    const float* in = X;
    for (int l = 0; l < 4; l++) {
        float* z = (l < 3) ? act + (size_t)(2 * l) * cap * H : Y;
        float* a = (l < 3) ? act + (size_t)(2 * l + 1) * cap * H : nullptr;
        dim3 g((dout[l] + 63) / 64, (n + 63) / 64);
        k_gemm<false, false><<<g, 256, 0, st>>>(n, dout[l], din[l], in, din[l], W[l], dout[l], z, dout[l], b[l], 0.f);
        if (l < 3) {
            k_silu<<<grid_for((size_t)n * H), 256, 0, st>>>(z, a, (size_t)n * H);
            in = a;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_contract_streamed(Plan& P, int n_rhs, cudaStream_t st) {
    const fbc_surrogate* S = P.sur;
    ContractArgs A = make_contract_args(P);
    A.tab32 = P.d_slice;
    A.kmul = 0;
    cudaError_t e = cudaSuccess;
    const int bs = 256;
    for (int k = 1; k < P.K && !e; k++) {
        if (P.n_far) {
            k_slice_features<<<(P.n_far + bs - 1) / bs, bs, 0, st>>>(P.d_far, P.n_far, k, P.L, P.c, P.d_sX);
            if ((e = surrogate_forward(S, S->d_pb, P.d_sX, P.n_far, P.d_sY, P.d_sact, P.n_far, st))) break;
            k_slice_far<<<(P.n_far + bs - 1) / bs, bs, 0, st>>>(P.d_far, P.n_far, k, P.L, P.c, P.d_sY, P.d_slice, P.Dx,
                                                                  P.box_x0, P.box_y0);
        }
        if (P.n_near)
            k_slice_near<<<(P.n_near + bs - 1) / bs, bs, 0, st>>>(P.d_near, P.n_near, k, P.d_near32, P.Dx, P.box_x0,
                                                                    P.box_y0, P.d_slice);
        if ((e = cudaGetLastError())) break;
        e = launch_contract_modes(P, A, k, 1, n_rhs, st);
    }
    return e;
}

void release_surrogate_buffers(Plan& P) {
    void* bufs[] = {P.d_far, P.d_near, P.d_near32, P.d_slice, P.d_sX, P.d_sY, P.d_sact};
    for (void* b : bufs)
        if (b) cudaFree(b);
    P.d_far = P.d_near = nullptr;
    P.d_near32 = P.d_slice = P.d_sX = P.d_sY = P.d_sact = nullptr;
    P.n_far = P.n_near = 0;
    P.sur_bytes = 0;
}

}  // namespace fbc

namespace {

int sfail(int code, const char* msg) { return fbc::report_error(code, msg); }

int scuda(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return fbc::report_error(e == cudaErrorMemoryAllocation ? FBC_ERR_OOM : FBC_ERR_CUDA, buf);
}

// rows of one network evaluation: the GEMM grid's y extent is ceil(n / 64) <= 65535
constexpr int kMaxRows = 65535 * 64;

int ensure_cap(fbc_surrogate* S, int n) {
    if (n > kMaxRows) return sfail(FBC_ERR_INVALID_ARG, "more than 65535 * 64 rows in one evaluation");
    if (n <= S->cap) return FBC_OK;
    if (S->d_act) cudaFree(S->d_act), S->d_act = nullptr;
    // Z1 A1 Z2 A2 Z3 A3, Y, dY, and three gradient buffers T, B0, B1
    const size_t per = (size_t)n * (9 * S->width + 2 * 6);
    cudaError_t e = cudaMalloc((void**)&S->d_act, per * sizeof(float));
    if (e) return scuda(e, "surrogate scratch");
    S->cap = n;
    return FBC_OK;
}

// Loss and gradients of the mean-squared error on a batch (X [n][4], T [n][6]).
int loss_and_grad(fbc_surrogate* S, const float* X, const float* T, int n, cudaStream_t st, double* loss) {
    using namespace fbc;
    int s = ensure_cap(S, n);
    if (s) return s;
    const int H = S->width, cap = S->cap;
    float* act = S->d_act;
    float* Y = act + (size_t)6 * cap * H;
    float* dY = Y + (size_t)cap * kOut;
    float* Tb = dY + (size_t)cap * kOut;   // gradient with respect to a layer's input activations
    float* Bz[2] = {Tb + (size_t)cap * H, Tb + (size_t)2 * cap * H};  // gradients with respect to Z, alternating
    cudaError_t e = surrogate_forward(S, S->d_p, X, n, Y, act, cap, st);
    if (e) return scuda(e, "surrogate forward");
    const int nb = 64;
    k_mse<<<nb, 256, 0, st>>>(Y, T, dY, n * kOut, S->d_loss);
    const int din[4] = {4, H, H, H}, dout[4] = {H, H, H, kOut};
    const float* A_in[4] = {X, act + (size_t)1 * cap * H, act + (size_t)3 * cap * H, act + (size_t)5 * cap * H};
    const float* Zs[3] = {act, act + (size_t)2 * cap * H, act + (size_t)4 * cap * H};
    const float* dcur = dY;  // gradient with respect to the current layer's output (pre-activation)
    for (int l = 3; l >= 0; l--) {
        float* dW = S->d_g + S->off[2 * l];
        float* db = S->d_g + S->off[2 * l + 1];
        dim3 gw((dout[l] + 63) / 64, (din[l] + 63) / 64);
        k_gemm<true, false><<<gw, 256, 0, st>>>(din[l], dout[l], n, A_in[l], din[l], dcur, dout[l], dW, dout[l], nullptr, 0.f);
        k_colsum<<<(dout[l] + 127) / 128, 128, 0, st>>>(dcur, n, dout[l], db);
        if (l > 0) {
            const float* Wl = S->d_p + S->off[2 * l];
            dim3 gx((din[l] + 63) / 64, (n + 63) / 64);
            k_gemm<false, true><<<gx, 256, 0, st>>>(n, din[l], dout[l], dcur, dout[l], Wl, dout[l], Tb, din[l], nullptr, 0.f);
            float* out = Bz[l & 1];
            k_silu_back<<<grid_for((size_t)n * H), 256, 0, st>>>(Zs[l - 1], Tb, out, (size_t)n * H);
            dcur = out;
        }
    }
    if ((e = cudaGetLastError())) return scuda(e, "surrogate backward");
    if (loss) {
        std::vector<double> part(nb);
        if ((e = cudaMemcpyAsync(part.data(), S->d_loss, nb * sizeof(double), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st)))
            return scuda(e, "loss readback");
        double t = 0.0;
        for (double p : part) t += p;
        *loss = t / (double)(n * kOut);
    }
    return FBC_OK;
}

}  // namespace

extern "C" {

int fbc_surrogate_create(int32_t width, uint64_t seed, fbc_surrogate** out) {
    fbc::report_error(FBC_OK, "");
    if (!out) return sfail(FBC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (width < 8 || width > 1024 || (width % 8)) return sfail(FBC_ERR_INVALID_ARG, "width must be a multiple of 8 in [8, 1024]");
    fbc_surrogate* S = new (std::nothrow) fbc_surrogate();
    if (!S) return sfail(FBC_ERR_OOM, "host allocation failed");
    S->width = width;
    const int H = width;
    const int sizes[8] = {4 * H, H, H * H, H, H * H, H, H * 6, 6};
    int o = 0;
    for (int t = 0; t < 8; t++) S->off[t] = o, o += sizes[t];
    S->n_params = o;
    // He-style initialisation from a seeded host generator (deterministic on every host)
    std::vector<float> p(o, 0.0f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    const int fan_in[4] = {4, H, H, H};
    for (int l = 0; l < 4; l++) {
        const double sd = std::sqrt(2.0 / fan_in[l]) * (l == 3 ? 0.1 : 1.0);
        for (int t = 0; t < sizes[2 * l]; t++) p[S->off[2 * l] + t] = (float)(sd * nd(rng));
    }
    cudaError_t e = cudaSuccess;
    float** bufs[5] = {&S->d_p, &S->d_pb, &S->d_g, &S->d_m, &S->d_v};
    for (auto b : bufs)
        if (!e) e = cudaMalloc((void**)b, sizeof(float) * o);
    if (!e) e = cudaMalloc((void**)&S->d_loss, 64 * sizeof(double));
    if (!e) e = cudaMemcpy(S->d_p, p.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(S->d_m, 0, sizeof(float) * o);
    if (!e) e = cudaMemset(S->d_v, 0, sizeof(float) * o);
    if (e) {
        int s = scuda(e, "surrogate allocation");
        fbc_surrogate_destroy(S);
        return s;
    }
    *out = S;
    return FBC_OK;
}

int fbc_surrogate_n_params(const fbc_surrogate* S) { return S ? S->n_params : 0; }

int fbc_surrogate_params(fbc_surrogate* S, float* host_out, const float* host_in) {
    fbc::report_error(FBC_OK, "");
    if (!S) return sfail(FBC_ERR_INVALID_ARG, "surrogate is NULL");
    cudaError_t e = cudaSuccess;
    if (host_in) e = cudaMemcpy(S->d_p, host_in, sizeof(float) * S->n_params, cudaMemcpyHostToDevice);
    if (!e && host_out) e = cudaMemcpy(host_out, S->d_p, sizeof(float) * S->n_params, cudaMemcpyDeviceToHost);
    return e ? scuda(e, "parameter copy") : FBC_OK;
}

int fbc_surrogate_forward(fbc_surrogate* S, const float* x, float* y, int32_t n, int32_t bf16_weights, void* stream) {
    fbc::report_error(FBC_OK, "");
    if (!S || !x || !y || n < 1) return sfail(FBC_ERR_INVALID_ARG, "bad arguments");
    int s = ensure_cap(S, n);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const float* params = S->d_p;
    if (bf16_weights) {
        fbc::k_round_bf16<<<fbc::grid_for(S->n_params), 256, 0, st>>>(S->d_p, S->d_pb, S->n_params);
        params = S->d_pb;
    }
    cudaError_t e = fbc::surrogate_forward(S, params, x, n, y, S->d_act, S->cap, st);
    return e ? scuda(e, "surrogate forward") : FBC_OK;
}

int fbc_surrogate_loss_grad(fbc_surrogate* S, const float* x, const float* t, int32_t n, double* loss, float* host_grad,
                            void* stream) {
    fbc::report_error(FBC_OK, "");
    if (!S || !x || !t || n < 1) return sfail(FBC_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    int s = loss_and_grad(S, x, t, n, st, loss);
    if (s) return s;
    if (host_grad) {
        cudaError_t e = cudaMemcpyAsync(host_grad, S->d_g, sizeof(float) * S->n_params, cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaStreamSynchronize(st);
        if (e) return scuda(e, "gradient readback");
    }
    return FBC_OK;
}

int fbc_surrogate_train(fbc_surrogate* S, const fbc_plan* plan, int32_t n_samples, double r_min, int32_t epochs,
                        int32_t batch, double lr, uint64_t seed, void* stream, double* final_loss) {
    fbc::report_error(FBC_OK, "");
    if (!S || !plan) return sfail(FBC_ERR_INVALID_ARG, "surrogate or plan is NULL");
    const fbc::Plan& P = plan->p;
    if (!P.tabulated || !P.d_table) return sfail(FBC_ERR_NOT_TABULATED, "the plan's exact table trains the surrogate");
    if (n_samples < 1 || epochs < 1 || batch < 1 || !(lr > 0.0) || !(r_min > 0.0))
        return sfail(FBC_ERR_INVALID_ARG, "bad training arguments");
    if (P.K < 2) return sfail(FBC_ERR_INVALID_ARG, "the surrogate models modes k >= 1 (L >= 2)");
    // far differences
    std::vector<int2> used(P.n_used);
    cudaError_t e = cudaMemcpy(used.data(), P.d_used, sizeof(int2) * P.n_used, cudaMemcpyDeviceToHost);
    if (e) return scuda(e, "used list");
    std::vector<int> far;
    for (int i = 0; i < P.n_used; i++)
        if ((double)used[i].x * used[i].x + (double)used[i].y * used[i].y >= r_min * r_min) far.push_back(i);
    if (far.empty()) return sfail(FBC_ERR_INVALID_ARG, "no differences at or beyond r_min");
    // (d, k) uniform over the far differences and the modes with q r <= cut
    const double q1 = 2.0 * M_PI / (P.L * P.c);
    double r_far_min = 1e300;
    for (int i : far) r_far_min = std::min(r_far_min, std::sqrt((double)used[i].x * used[i].x + (double)used[i].y * used[i].y));
    if (q1 * r_far_min > fbc::kQrCut) return sfail(FBC_ERR_INVALID_ARG, "every far pair is beyond the q r cut");
    std::mt19937_64 rng(seed);
    std::vector<int> sd(n_samples), sk(n_samples);
    for (int i = 0; i < n_samples;) {
        const int di = far[rng() % far.size()];
        const int k = 1 + (int)(rng() % (uint64_t)(P.K - 1));
        const double r = std::sqrt((double)used[di].x * used[di].x + (double)used[di].y * used[di].y);
        if (q1 * k * r > fbc::kQrCut) continue;
        sd[i] = di, sk[i] = k, i++;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int *d_sd = nullptr, *d_sk = nullptr;
    float *d_X = nullptr, *d_T = nullptr;
    e = cudaMalloc((void**)&d_sd, sizeof(int) * n_samples);
    if (!e) e = cudaMalloc((void**)&d_sk, sizeof(int) * n_samples);
    if (!e) e = cudaMalloc((void**)&d_X, sizeof(float) * 4 * (size_t)n_samples);
    if (!e) e = cudaMalloc((void**)&d_T, sizeof(float) * 6 * (size_t)n_samples);
    if (!e) e = cudaMemcpy(d_sd, sd.data(), sizeof(int) * n_samples, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(d_sk, sk.data(), sizeof(int) * n_samples, cudaMemcpyHostToDevice);
    int status = FBC_OK;
    if (!e) {
        fbc::k_samples<<<(n_samples + 255) / 256, 256, 0, st>>>(P.d_used, d_sd, d_sk, n_samples, P.d_table, P.Dx, P.Dy,
                                                              P.box_x0, P.box_y0, P.L, P.c, d_X, d_T);
        e = cudaGetLastError();
    }
    double loss = 0.0;
    const int nb = (n_samples + batch - 1) / batch;
    for (int ep = 0; ep < epochs && !e && status == FBC_OK; ep++) {
        // cosine-decayed learning rate
        const double lr_ep = lr * 0.5 * (1.0 + std::cos(M_PI * ep / (double)epochs));
        double ep_loss = 0.0;
        for (int bi = 0; bi < nb && status == FBC_OK; bi++) {
            const int i0 = bi * batch, n = std::min(batch, n_samples - i0);
            const bool last = (bi == nb - 1);
            double bl = 0.0;
            status = loss_and_grad(S, d_X + (size_t)i0 * 4, d_T + (size_t)i0 * 6, n, st, last ? &bl : nullptr);
            if (status) break;
            S->step++;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - std::pow(b1, (float)S->step), c2 = 1.f - std::pow(b2, (float)S->step);
            fbc::k_adam<<<fbc::grid_for(S->n_params), 256, 0, st>>>(S->d_p, S->d_g, S->d_m, S->d_v, S->n_params,
                                                                    (float)lr_ep, b1, b2, c1, c2, 1e-8f);
            if (last) ep_loss = bl;
        }
        loss = ep_loss;
        e = cudaGetLastError();
    }
    cudaFree(d_sd), cudaFree(d_sk), cudaFree(d_X), cudaFree(d_T);
    if (status) return status;
    if (e) return scuda(e, "surrogate training");
    if (final_loss) *final_loss = loss;
    return FBC_OK;
}

int fbc_surrogate_eval_table(fbc_surrogate* S, const fbc_plan* plan, const int32_t* d, const int32_t* k, int32_t n,
                             double* out) {
    fbc::report_error(FBC_OK, "");
    if (!S || !plan || !d || !k || !out || n < 1) return sfail(FBC_ERR_INVALID_ARG, "bad arguments");
    const fbc::Plan& P = plan->p;
    // features on the host (same formula as the device kernels), network on the device
    std::vector<float> X(4 * (size_t)n);
    for (int i = 0; i < n; i++) {
        const double r = std::sqrt((double)d[2 * i] * d[2 * i] + (double)d[2 * i + 1] * d[2 * i + 1]);
        if (!(r > 0.0) || k[i] < 1 || k[i] >= P.K) return sfail(FBC_ERR_INVALID_ARG, "need d != 0 and 1 <= k < K");
        const double qr = 2.0 * M_PI * k[i] / (P.L * P.c) * r;
        X[4 * i + 0] = (float)(qr / 32.0), X[4 * i + 1] = (float)(d[2 * i] / r), X[4 * i + 2] = (float)(d[2 * i + 1] / r);
        X[4 * i + 3] = (float)(std::log(r) / 5.0);
    }
    float *d_X = nullptr, *d_Y = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_X, sizeof(float) * 4 * (size_t)n);
    if (!e) e = cudaMalloc((void**)&d_Y, sizeof(float) * 6 * (size_t)n);
    if (!e) e = cudaMemcpy(d_X, X.data(), sizeof(float) * 4 * (size_t)n, cudaMemcpyHostToDevice);
    int s = e ? scuda(e, "eval buffers") : fbc_surrogate_forward(S, d_X, d_Y, n, 1, nullptr);
    std::vector<float> Y(6 * (size_t)n);
    if (!s) {
        e = cudaMemcpy(Y.data(), d_Y, sizeof(float) * 6 * (size_t)n, cudaMemcpyDeviceToHost);
        if (e) s = scuda(e, "eval readback");
    }
    cudaFree(d_X), cudaFree(d_Y);
    if (s) return s;
    for (int i = 0; i < n; i++) {
        const double r = std::sqrt((double)d[2 * i] * d[2 * i] + (double)d[2 * i + 1] * d[2 * i + 1]);
        const double qr = 2.0 * M_PI * k[i] / (P.L * P.c) * r;
        const double sc = qr > fbc::kQrCut ? 0.0 : std::exp(-qr) / (P.c * std::sqrt(1.0 + qr));
        for (int j = 0; j < 6; j++) out[6 * (size_t)i + j] = Y[6 * (size_t)i + j] * sc;
    }
    return FBC_OK;
}

int fbc_plan_attach_surrogate(fbc_plan* plan, fbc_surrogate* S, double r_min, int32_t release_tables) {
    fbc::report_error(FBC_OK, "");
    if (!plan) return sfail(FBC_ERR_INVALID_ARG, "plan is NULL");
    fbc::Plan& P = plan->p;
    if (P.host_only) return sfail(FBC_ERR_INVALID_ARG, "host-only plan");
    if (!S) {
        if (P.tables_released) return sfail(FBC_ERR_INVALID_ARG, "tables were released: the surrogate cannot be detached");
        cudaDeviceSynchronize();
        fbc::release_surrogate_buffers(P);
        P.sur = nullptr;
        return FBC_OK;
    }
    if (!P.tabulated || P.tables_released) return sfail(FBC_ERR_NOT_TABULATED, "attach needs the exact tables");
    if (!(r_min > 0.0)) return sfail(FBC_ERR_INVALID_ARG, "r_min must be positive");
    if (P.precision != FBC_PREC_FP32 && !fbc::is_tensor_precision(P.precision))
        return sfail(FBC_ERR_UNSUPPORTED, "the surrogate serves the FP32 and tensor-core precisions");
    cudaDeviceSynchronize();
    fbc::release_surrogate_buffers(P);
    std::vector<int2> used(P.n_used), far, near;
    cudaError_t e = cudaMemcpy(used.data(), P.d_used, sizeof(int2) * P.n_used, cudaMemcpyDeviceToHost);
    if (e) return scuda(e, "used list");
    for (const int2& d : used) ((double)d.x * d.x + (double)d.y * d.y >= r_min * r_min ? far : near).push_back(d);
    if (far.size() > (size_t)kMaxRows) return sfail(FBC_ERR_UNSUPPORTED, "more than 65535 * 64 far differences");
    P.n_far = (int)far.size(), P.n_near = (int)near.size();
    const size_t cells = (size_t)P.Dy * P.Dx;
    size_t bytes_total = 0;
    auto A = [&](void** p, size_t bytes) {
        bytes = std::max<size_t>(bytes, 16);
        if (!e) e = cudaMalloc(p, bytes);
        if (!e) bytes_total += bytes;
    };
    A((void**)&P.d_far, sizeof(int2) * far.size());
    A((void**)&P.d_near, sizeof(int2) * near.size());
    A((void**)&P.d_near32, sizeof(float) * 6 * near.size() * P.K);
    A((void**)&P.d_slice, sizeof(float) * 6 * cells);
    A((void**)&P.d_sX, sizeof(float) * 4 * far.size());
    A((void**)&P.d_sY, sizeof(float) * 6 * far.size());
    A((void**)&P.d_sact, sizeof(float) * 6 * far.size() * S->width);
    if (!e && !far.empty()) e = cudaMemcpy(P.d_far, far.data(), sizeof(int2) * far.size(), cudaMemcpyHostToDevice);
    if (!e && !near.empty()) e = cudaMemcpy(P.d_near, near.data(), sizeof(int2) * near.size(), cudaMemcpyHostToDevice);
    // cells no pair reads stay zero (padding columns multiply them by zero forces)
    if (!e) e = cudaMemset(P.d_slice, 0, sizeof(float) * 6 * cells);
    if (!e && !near.empty()) {
        const size_t t = (size_t)near.size() * P.K;
        fbc::k_near_gather<<<(unsigned)((t + 255) / 256), 256>>>(P.d_near, (int)near.size(), P.K, P.d_table, P.Dx, P.Dy,
                                                                  P.box_x0, P.box_y0, P.d_near32);
        e = cudaGetLastError();
    }
    if (!e) {
        fbc::k_round_bf16<<<fbc::grid_for(S->n_params), 256>>>(S->d_p, S->d_pb, S->n_params);
        e = cudaGetLastError();
    }
    if (!e) e = cudaDeviceSynchronize();
    if (e) {
        fbc::release_surrogate_buffers(P);
        return scuda(e, "attach");
    }
    P.sur = S;
    P.sur_rmin = r_min;
    P.sur_bytes = bytes_total;
    if (release_tables) {
        // the k = 0 double-float slice stays; the K-slice tables go
        const size_t kcells = (size_t)P.K * cells;
        if (P.d_table) cudaFree(P.d_table), P.d_table = nullptr;
        if (P.d_table32) cudaFree(P.d_table32), P.d_table32 = nullptr, P.workspace_bytes -= kcells * 6 * sizeof(float);
        if (P.d_table_x2) cudaFree(P.d_table_x2), P.d_table_x2 = nullptr, P.workspace_bytes -= kcells * 12 * sizeof(float);
        P.tables_released = true;
        P.table_bytes = 0;
    }
    return FBC_OK;
}

void fbc_surrogate_destroy(fbc_surrogate* S) {
    if (!S) return;
    void* bufs[] = {S->d_p, S->d_pb, S->d_g, S->d_m, S->d_v, S->d_act, S->d_loss};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete S;
}

}  // extern "C"
