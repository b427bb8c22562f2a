// Learned surrogate of the per-mode kernel table g^k(d) for far pairs.
//
// A multilayer perceptron 4 -> H -> H -> H -> 6 with SiLU activations maps the
// features of a (difference d, wavenumber k >= 1) pair,
//     x = (ln(q r) / 4, d_x / r, d_y / r, ln(r) / 5),   r = |d|,  q = 2 pi k / (L c),
// to the six independent reals of g^k(d) (Re g11, Re g12, Re g22, Re g33,
// Im g13, Im g23) divided by the smooth decay factor
//     s(q, r) = exp(-q r) / (c sqrt(1 + q r)),
// so that the targets are O(1) although the modes decay exponentially in q r.
// The Green function is homogeneous of degree -1, so for r well beyond the
// lattice spacing the mode entry depends on q r and the direction of d only
// (lattice corrections fall off like exp(-2 pi r / c)); ln(q r) makes the
// logarithm of the small-q r regime a linear function of an input.
// It is trained on the plan's own exact FP64 table (the tables the method
// itself generates) by the kernels of this file: a tiled FP32 GEMM used for
// the forward pass and both backward products, SiLU and its derivative, the
// mean-squared loss, bias reductions and Adam.  For inference the weights are
// rounded to bf16 values and the products accumulate in FP32 (fused
// tensor-core kernel in fbc_mlp_tc.cu).
//
// Use in the pad update: a plan in a CUDA-core FP32 or tensor-core precision
// streams its table a chunk of modes at a time: for modes k0 .. k0 + m - 1 the
// slices [m][Dy][Dx][6] are assembled from a compact exact copy for
// |d| < r_min (near field) and by the fused network for |d| >= r_min, and one
// contraction launch over those m modes reads them while they sit in L2; the
// K-slice tables need not exist.
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
    int* d_status = nullptr;   // error word of the fused inference kernel
};

namespace fbc {
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
    const double qr = surrogate_features(d.x, d.y, k, L, c, X + (size_t)i * kSurIn);
    const double inv_s = 1.0 / surrogate_scale(qr, c);
    const double* src = table + (((size_t)k * Dy + (d.y - box_y0)) * Dx + (d.x - box_x0)) * 6;
    for (int j = 0; j < 6; j++) T[(size_t)i * 6 + j] = (float)(src[j] * inv_s);
}

// Near entries of modes kbase .. kbase + n_modes - 1 copied into their slices
// from the compact exact table.
__global__ void k_slice_near(const int2* __restrict__ near, int n, int kbase, int n_modes,
                             const float* __restrict__ near32, int Dx, int box_x0, int box_y0, size_t slice_floats,
                             float* __restrict__ slice) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)n * n_modes) return;
    const int j = (int)(t / n), i = (int)(t % n);
    const int2 d = near[i];
    const size_t cell = (size_t)(d.y - box_y0) * Dx + (d.x - box_x0);
    const float* src = near32 + ((size_t)(kbase + j) * n + i) * 6;
    float* o = slice + (size_t)j * slice_floats + cell * 6;
    for (int e = 0; e < 6; e++) o[e] = src[e];
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

MlpArgs mlp_args(const fbc_surrogate* S, const float* params, int* status) {
    MlpArgs a;
    a.params = params;
    a.H = S->width;
    for (int t = 0; t < 8; t++) a.off[t] = S->off[t];
    a.status = status;
    return a;
}

cudaError_t launch_contract_streamed(Plan& P, int n_rhs, cudaStream_t st) {
    const fbc_surrogate* S = P.sur;
    ContractArgs A = make_contract_args(P);
    A.tab32 = P.d_slice;
    MlpArgs m = mlp_args(S, S->d_pb, P.d_status);
    m.far = P.d_far, m.n = P.n_far, m.L = P.L, m.c = P.c;
    m.slice = P.d_slice, m.Dx = P.Dx, m.box_x0 = P.box_x0, m.box_y0 = P.box_y0;
    m.slice_floats = (size_t)P.Dy * P.Dx * 6;
    cudaError_t e = cudaSuccess;
    for (int k0 = 1; k0 < P.K && !e; k0 += P.sur_chunk) {
        const int nm = std::min(P.sur_chunk, P.K - k0);
        if (P.n_far) {
            m.k0 = k0, m.n_modes = nm;
            if ((e = launch_mlp_tc(m, st))) break;
        }
        if (P.n_near) {
            const size_t t = (size_t)P.n_near * nm;
            k_slice_near<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(P.d_near, P.n_near, k0, nm, P.d_near32, P.Dx,
                                                                      P.box_x0, P.box_y0, m.slice_floats, P.d_slice);
        }
        if ((e = cudaGetLastError())) break;
        A.kbase = k0;
        e = launch_contract_modes(P, A, k0, nm, n_rhs, st);
    }
    return e;
}

void release_surrogate_buffers(Plan& P) {
    void* bufs[] = {P.d_far, P.d_near, P.d_near32, P.d_slice};
    for (void* b : bufs)
        if (b) cudaFree(b);
    P.d_far = P.d_near = nullptr;
    P.d_near32 = P.d_slice = nullptr;
    P.n_far = P.n_near = P.sur_chunk = 0;
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
    if (!e) e = cudaMalloc((void**)&S->d_status, sizeof(int));
    if (!e) e = cudaMemset(S->d_status, 0, sizeof(int));
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
        if (fbc::mlp_tc_supported(S->width)) {
            fbc::MlpArgs m = fbc::mlp_args(S, params, S->d_status);
            m.n = n, m.X = x, m.Y = y;
            cudaError_t e = fbc::launch_mlp_tc(m, st);
            return e ? scuda(e, "fused surrogate inference") : FBC_OK;
        }
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
    // d uniform over the far differences that have a mode below the q r cut;
    // k log-uniform over 1 .. kmax(d) (the modes with q r <= cut), which puts
    // as many samples in each octave of q r as the small-q r entries, the
    // largest ones, need
    const double q1 = 2.0 * M_PI / (P.L * P.c);
    std::vector<int> far_ok;
    std::vector<int> kmax;
    for (int i : far) {
        const double r = std::sqrt((double)used[i].x * used[i].x + (double)used[i].y * used[i].y);
        const int km = std::min(P.K - 1, (int)std::floor(fbc::kQrCut / (q1 * r)));
        if (km >= 1) far_ok.push_back(i), kmax.push_back(km);
    }
    if (far_ok.empty()) return sfail(FBC_ERR_INVALID_ARG, "every far pair is beyond the q r cut");
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> u01(0.0, 1.0);
    std::vector<int> sd(n_samples), sk(n_samples);
    for (int i = 0; i < n_samples; i++) {
        const size_t j = rng() % far_ok.size();
        const int k = (int)std::floor(std::exp(u01(rng) * std::log(kmax[j] + 1.0)));
        sd[i] = far_ok[j], sk[i] = std::min(std::max(k, 1), kmax[j]);
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
    // features on the host (the function the device kernels use), network on the device
    std::vector<float> X(4 * (size_t)n);
    std::vector<double> sc(n);
    for (int i = 0; i < n; i++) {
        if ((d[2 * i] == 0 && d[2 * i + 1] == 0) || k[i] < 1 || k[i] >= P.K)
            return sfail(FBC_ERR_INVALID_ARG, "need d != 0 and 1 <= k < K");
        sc[i] = fbc::surrogate_scale(fbc::surrogate_features(d[2 * i], d[2 * i + 1], k[i], P.L, P.c, &X[4 * (size_t)i]),
                                     P.c);
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
    int st = 0;
    if (cudaMemcpy(&st, S->d_status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && st) {
        cudaMemset(S->d_status, 0, sizeof(int));
        return sfail(st, "fused surrogate inference timed out");
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 6; j++) out[6 * (size_t)i + j] = Y[6 * (size_t)i + j] * sc[i];
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
    if (!fbc::mlp_tc_supported(S->width))
        return sfail(FBC_ERR_UNSUPPORTED, "the fused inference kernel takes widths 32, 64, 96 and 128");
    cudaDeviceSynchronize();
    fbc::release_surrogate_buffers(P);
    std::vector<int2> used(P.n_used), far, near;
    cudaError_t e = cudaMemcpy(used.data(), P.d_used, sizeof(int2) * P.n_used, cudaMemcpyDeviceToHost);
    if (e) return scuda(e, "used list");
    for (const int2& d : used) ((double)d.x * d.x + (double)d.y * d.y >= r_min * r_min ? far : near).push_back(d);
    if (far.size() > (size_t)kMaxRows) return sfail(FBC_ERR_UNSUPPORTED, "more than 65535 * 64 far differences");
    P.n_far = (int)far.size(), P.n_near = (int)near.size();
    const size_t cells = (size_t)P.Dy * P.Dx;
    // modes per chunk: their slices (about 48 MB together) stay in L2 between
    // the network that writes them and the contraction that reads them
    const size_t slice_bytes = cells * 6 * sizeof(float);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>({(size_t)32, (size_t)std::max(1, P.K - 1),
                                                                  ((size_t)48 << 20) / slice_bytes}));
    size_t bytes_total = 0;
    auto A = [&](void** p, size_t bytes) {
        bytes = std::max<size_t>(bytes, 16);
        if (!e) e = cudaMalloc(p, bytes);
        if (!e) bytes_total += bytes;
    };
    A((void**)&P.d_far, sizeof(int2) * far.size());
    A((void**)&P.d_near, sizeof(int2) * near.size());
    A((void**)&P.d_near32, sizeof(float) * 6 * near.size() * P.K);
    A((void**)&P.d_slice, slice_bytes * chunk);
    if (!e && !far.empty()) e = cudaMemcpy(P.d_far, far.data(), sizeof(int2) * far.size(), cudaMemcpyHostToDevice);
    if (!e && !near.empty()) e = cudaMemcpy(P.d_near, near.data(), sizeof(int2) * near.size(), cudaMemcpyHostToDevice);
    // cells no pair reads stay zero (padding columns multiply them by zero forces)
    if (!e) e = cudaMemset(P.d_slice, 0, slice_bytes * chunk);
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
    P.sur_chunk = chunk;
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

int fbc_surrogate_sync_status(fbc_surrogate* S, void* stream) {
    fbc::report_error(FBC_OK, "");
    if (!S) return sfail(FBC_ERR_INVALID_ARG, "surrogate is NULL");
    int st = 0;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (!e) e = cudaMemcpy(&st, S->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e) return scuda(e, "surrogate status");
    if (st) {
        cudaMemset(S->d_status, 0, sizeof(int));
        return sfail(st, "fused surrogate inference timed out");
    }
    return FBC_OK;
}

void fbc_surrogate_destroy(fbc_surrogate* S) {
    if (!S) return;
    void* bufs[] = {S->d_p, S->d_pb, S->d_g, S->d_m, S->d_v, S->d_act, S->d_loss, S->d_status};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete S;
}

}  // extern "C"
