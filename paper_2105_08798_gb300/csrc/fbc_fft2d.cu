// In-plane FFT forms of the per-mode contraction (FBC_PREC_FFT64: FP64
// throughout; FBC_PREC_FFT32: FP32 transforms and kernel for k >= 1, the
// k = 0 mode on the FP64 transforms).
//
// The dense contraction evaluates, for every wavenumber k and right-hand side,
//     U(a) = sum_b M^k(x_a - x_b) z(b),
// where z(b) = x(b) + i y'(b) packs the two real 3-vectors of the six-vector
// form into one complex 3-vector and M^k(d) is the real 3x3 matrix built from
// the six table reals,
//     M = [[a11, a12, -b13], [a12, a22, -b23], [b13, b23, a33]].
// Because the kernel depends only on the lattice difference d (translation
// invariance of the Green function in the plane, Sec. 3.1), this is a 2D
// convolution over the lattice.  It is evaluated exactly by a circular
// convolution on an Mx x My grid with at least 2 max|d| + 1 points per side
// (each side 2^a 3^b 5^c, the cheapest such length): every difference d that
// occurs, and its mirror -d, then has a residue of its own, so the circular
// sum at a pad site picks up exactly the terms of the direct sum.  The kernel is placed at d with the table values
// and at -d with the exact mirror relations of the Green function (a_ij even
// and b_i3 odd in d), which makes its 2D DFT the Hermitian matrix
//     Mhat = [[A11, A12, -i B13], [A12, A22, -i B23], [i B13, i B23, A33]]
// with six real fields A11, A12, A22, A33 (the DFTs of the even a_ij) and
// B13, B23 (DFT(b_i3) = i B_i3); they are computed once per plan.
//
// One apply, per (right-hand side, mode) item:
//   P1  gather z of every interface row onto its grid row, forward FFT along x
//       (only the rows that hold interface sites);
//   P2  per grid column: forward FFT along y, multiply by Mhat, inverse FFT
//       along y; keep only the rows that hold pad sites;
//   P3  inverse FFT along x of every pad row, scale by 1/(Mx My) and scatter
//       the pad sites into uh.
// Transforms in shared memory in the Stockham form (natural order in and
// out, two buffers used in turn): each pass gives every thread one
// sub-transform of radix 8, 6, 5, 4, 3 or 2 in registers; the lengths are
// chosen for the fewest passes (216 = 6 x 6 x 6, 320 = 5 x 8 x 8: three
// passes through shared memory each).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <map>
#include <set>
#include <vector>

#include "fbc_fft.cuh"
#include "fbc_internal.cuh"

namespace fbc {

struct FftGrid {
    int Mx = 0, My = 0;
    Fft1D fx, fy;
    int ny_i = 0, ny_p = 0;
    int Q = 0;                     // (rhs, mode) items per chunk of the workspace
    int* d_row_i = nullptr;        // [ny_i + 1] CSR of the interface rows
    int2* d_ent_i = nullptr;       // (x position on the grid | row << 12, fh slot)
    int* d_row_p = nullptr;        // [ny_p + 1]
    int2* d_ent_p = nullptr;       // (x position on the grid | row << 12, uh slot)
    int* d_ypos_i = nullptr;       // [ny_i] y position on the grid of each interface row
    int* d_ypos_p = nullptr;       // [ny_p]
    double2* d_twx = nullptr;      // [Mx] exp(-2 pi i j / Mx)
    double2* d_twy = nullptr;      // [My]
    double* d_mhat = nullptr;      // [K][Mx][My][6]: A11 A12 A22 A33 B13 B23
    float* d_mhat32 = nullptr;     // the same rounded to FP32 (FBC_PREC_FFT32)
    float2* d_twx32 = nullptr;     // twiddles rounded to FP32
    float2* d_twy32 = nullptr;
    double2* d_T1 = nullptr;       // [Q][Mx][ny_i][3] (2Q items when complex FP32)
    double2* d_T2 = nullptr;       // [Q][Mx][ny_p][3]
    int2* d_used = nullptr;        // [n_used] differences placed on the grid (table entries)
    unsigned char* d_mirror = nullptr;  // [n_used] 1: also place the mirror -d (it is not a table entry)
    int n_used = 0;
    size_t bytes = 0;
};

namespace {

using namespace fft;

constexpr int kFftThreads = 384;  // one radix-8 work item per thread when a block holds 3 x 1024 points
constexpr int kSetupThreads = 256;
constexpr int kRowElems = 1024;  // complex elements per component a block of P1 / P3 transforms

// the cheapest length >= need (cost: points x (passes + 1)), and its passes
Fft1D choose_length(int need) {
    Fft1D F;
    long long best_cost = -1;
    std::vector<int> best;
    for (int N = std::max(2, need); N <= std::max(4, 2 * need); N++) {
        std::vector<int> p = radix_passes(N);
        if (p.empty() || (int)p.size() > kMaxPass) continue;
        const long long cost = (long long)N * (long long)(p.size() + 1);
        if (best_cost < 0 || cost < best_cost) best_cost = cost, best = p, F.N = N;
    }
    F.np = (int)best.size();
    int Ns = 1;
    for (int q = 0; q < F.np; q++) {
        F.R[q] = best[q], F.Ns[q] = Ns, F.NR[q] = F.N / best[q], F.tstep[q] = F.N / (Ns * best[q]);
        div_magic(F.NR[q], &F.mNR[q], &F.lNR[q]);
        div_magic(Ns, &F.mNs[q], &F.lNs[q]);
        Ns *= best[q];
    }
    return F;
}


template <typename R> struct CxOf;
template <> struct CxOf<float> { using T = float2; };
template <> struct CxOf<double> { using T = double2; };
template <typename R> using Cx = typename CxOf<R>::T;

// Items are (rhs, mode) pairs in mode-major order, item = k * R + r, so that the items of one
// workspace chunk share few modes and each mode's Mhat slice is read from L2 by all its rhs.
struct FftArgs {
    const double* fh;
    double* uh;
    const void* mhat;  // [K][Mx][My][6] of the transform's real type
    void* T1;          // [Q][Mx][ny_i][3] complex
    void* T2;          // [Q][Mx][ny_p][3] complex
    const int* row_i;
    const int2* ent_i;
    const int* row_p;
    const int2* ent_p;
    const int* ypos_i;
    const int* ypos_p;
    const void* twx;
    const void* twy;
    Fft1D fx, fy;
    int Mx, My, ny_i, ny_p, R, K, NIpad, NPpad, item0;
    double scale;
    // divisions of the index decodes: by the rows per block of P1 / P3, ny_i, ny_p and My
    unsigned mG, mNyi, mNyp, mMy;
    int lG, lNyi, lNyp, lMy;
};

// P1: rows of interface sites, forward FFT along x.  Block: G rows of one item.
template <typename R>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 ? 3 : 2) k_fft_rows_fwd(FftArgs A, int G) {
    using C = Cx<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = (C*)smraw;  // [G][3][Mx] (padded index), then the same again as scratch
    const int iq = blockIdx.y, item = A.item0 + iq, k = item / A.R, r = item - k * A.R;
    const int row0 = blockIdx.x * G, n = padded(G * 3 * A.Mx);
    for (int t = threadIdx.x; t < n; t += blockDim.x) s[t] = mkc<C>(0, 0);
    __syncthreads();
    const double* fk = A.fh + ((size_t)r * A.K + k) * A.NIpad * 6;
    // all entries of the block's rows in one loop (each entry carries its row)
    const int e1 = A.row_i[min(row0 + G, A.ny_i)];
    for (int e = A.row_i[row0] + threadIdx.x; e < e1; e += blockDim.x) {
        const int2 en = A.ent_i[e];
        const int g = (en.x >> 12) - row0, xp = en.x & 4095;
        const double* v = fk + (size_t)en.y * 6;
        for (int c = 0; c < 3; c++) s[sx((g * 3 + c) * A.Mx + xp)] = mkc<C>((R)v[c], (R)v[3 + c]);
    }
    __syncthreads();
    const C* res = fft_smem<false>(s, s + n, G * 3, A.fx, (const C*)A.twx);
    const int gr = min(G, A.ny_i - row0);
    C* out = (C*)A.T1 + (size_t)iq * A.Mx * A.ny_i * 3;
    for (int t = threadIdx.x; t < A.Mx * G * 3; t += blockDim.x) {
        const int q = t / 3, c = t - 3 * q, xi = fdiv(q, A.mG, A.lG), g = q - xi * G;
        if (g < gr) out[((size_t)xi * A.ny_i + row0 + g) * 3 + c] = res[sx((g * 3 + c) * A.Mx + xi)];
    }
}

// P2: G grid columns of one item: forward FFT along y, Mhat, inverse FFT along y, pad rows out.
template <typename R>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 ? 3 : 2) k_fft_cols(FftArgs A, int G) {
    using C = Cx<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = (C*)smraw;  // [G][3][My] (padded index), then the same again as scratch
    const int iq = blockIdx.y, item = A.item0 + iq, k = item / A.R;
    const int xi0 = blockIdx.x * G, gc = min(G, A.Mx - xi0), n = padded(G * 3 * A.My);
    for (int t = threadIdx.x; t < n; t += blockDim.x) s[t] = mkc<C>(0, 0);
    __syncthreads();
    const C* in = (const C*)A.T1 + (size_t)iq * A.Mx * A.ny_i * 3;
    for (int t = threadIdx.x; t < gc * A.ny_i * 3; t += blockDim.x) {
        const int q = t / 3, c = t - 3 * q, g = fdiv(q, A.mNyi, A.lNyi), row = q - g * A.ny_i;
        s[sx((g * 3 + c) * A.My + A.ypos_i[row])] = in[((size_t)(xi0 + g) * A.ny_i + row) * 3 + c];
    }
    __syncthreads();
    C* z0p = fft_smem<false>(s, s + n, G * 3, A.fy, (const C*)A.twy);
    for (int t = threadIdx.x; t < gc * A.My; t += blockDim.x) {
        const int g = fdiv(t, A.mMy, A.lMy), et = t - g * A.My;
        const R* m = (const R*)A.mhat + (((size_t)k * A.Mx + xi0 + g) * A.My + et) * 6;
        const R a11 = m[0], a12 = m[1], a22 = m[2], a33 = m[3], b13 = m[4], b23 = m[5];
        const int i0 = sx(g * 3 * A.My + et), i1 = sx((g * 3 + 1) * A.My + et), i2 = sx((g * 3 + 2) * A.My + et);
        const C z0 = z0p[i0], z1 = z0p[i1], z2 = z0p[i2];
        // (-i b) z = (b z.y, -b z.x),  (i b) z = (-b z.y, b z.x)
        z0p[i0] = mkc<C>(fmx(a11, z0.x, fmx(a12, z1.x, b13 * z2.y)), fmx(a11, z0.y, fmx(a12, z1.y, -b13 * z2.x)));
        z0p[i1] = mkc<C>(fmx(a12, z0.x, fmx(a22, z1.x, b23 * z2.y)), fmx(a12, z0.y, fmx(a22, z1.y, -b23 * z2.x)));
        z0p[i2] = mkc<C>(fmx(a33, z2.x, -fmx(b13, z0.y, b23 * z1.y)), fmx(a33, z2.y, fmx(b13, z0.x, b23 * z1.x)));
    }
    __syncthreads();
    const C* res = fft_smem<true>(z0p, z0p == s ? s + n : s, G * 3, A.fy, (const C*)A.twy);
    C* out = (C*)A.T2 + (size_t)iq * A.Mx * A.ny_p * 3;
    for (int t = threadIdx.x; t < gc * A.ny_p * 3; t += blockDim.x) {
        const int q = t / 3, c = t - 3 * q, g = fdiv(q, A.mNyp, A.lNyp), row = q - g * A.ny_p;
        out[((size_t)(xi0 + g) * A.ny_p + row) * 3 + c] = res[sx((g * 3 + c) * A.My + A.ypos_p[row])];
    }
}

// P3: G pad rows of one item: inverse FFT along x, scale, scatter the pad sites into uh.
template <typename R>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 ? 3 : 2) k_fft_rows_inv(FftArgs A, int G) {
    using C = Cx<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* s = (C*)smraw;  // [G][3][Mx] (padded index), then the same again as scratch
    const int iq = blockIdx.y, item = A.item0 + iq, k = item / A.R, r = item - k * A.R;
    const int row0 = blockIdx.x * G, gr = min(G, A.ny_p - row0), n = padded(G * 3 * A.Mx);
    const C* in = (const C*)A.T2 + (size_t)iq * A.Mx * A.ny_p * 3;
    for (int t = threadIdx.x; t < A.Mx * G * 3; t += blockDim.x) {
        const int q = t / 3, c = t - 3 * q, xi = fdiv(q, A.mG, A.lG), g = q - xi * G;
        s[sx((g * 3 + c) * A.Mx + xi)] = g < gr ? in[((size_t)xi * A.ny_p + row0 + g) * 3 + c] : mkc<C>(0, 0);
    }
    __syncthreads();
    const C* res = fft_smem<true>(s, s + n, G * 3, A.fx, (const C*)A.twx);
    double* uk = A.uh + ((size_t)r * A.K + k) * A.NPpad * 6;
    const int e1 = A.row_p[row0 + gr];
    for (int e = A.row_p[row0] + threadIdx.x; e < e1; e += blockDim.x) {
        const int2 en = A.ent_p[e];
        const int g = (en.x >> 12) - row0, xp = en.x & 4095;
        double* o = uk + (size_t)en.y * 6;
        for (int c = 0; c < 3; c++) {
            const C v = res[sx((g * 3 + c) * A.Mx + xp)];
            o[c] = (double)v.x * A.scale, o[3 + c] = (double)v.y * A.scale;
        }
    }
}

__global__ void k_fft_to_f32(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// ---- the kernel's transform (setup) ----------------------------------------

// place the six table fields of modes k0 .. k0 + nk - 1 on the grid: S [nk][6][My][Mx] complex (zeroed before)
__global__ void k_fft_place(const double* __restrict__ tab, const int2* __restrict__ used,
                            const unsigned char* __restrict__ mirror, int n_used, int k0, int nk, int Dx, int Dy,
                            int box_x0, int box_y0, int Mx, int My, double2* __restrict__ S) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_used * nk) return;
    const int u = (int)(t % n_used), kk = (int)(t / n_used);
    const int2 d = used[u];
    const double* v = tab + (((size_t)(k0 + kk) * Dy + (d.y - box_y0)) * Dx + (d.x - box_x0)) * 6;
    const int px = ((d.x % Mx) + Mx) % Mx, py = ((d.y % My) + My) % My;
    const int qx = (Mx - px) % Mx, qy = (My - py) % My;
    double2* base = S + (size_t)kk * 6 * My * Mx;
    for (int f = 0; f < 6; f++) {
        base[((size_t)f * My + py) * Mx + px] = make_double2(v[f], 0.0);
        if (mirror[u]) base[((size_t)f * My + qy) * Mx + qx] = make_double2(f < 4 ? v[f] : -v[f], 0.0);
    }
}

// forward FFT along x of G rows (of length Mx) of one field per block, in place in global memory;
// S holds nf fields of My rows each, block (bx, f) takes rows bx G .. bx G + G - 1 of field f
__global__ void __launch_bounds__(kSetupThreads) k_fft_dense_rows(double2* S, int Mx, int My, Fft1D fx, int G,
                                                                   const double2* __restrict__ twx) {
    extern __shared__ double2 sd[];  // [G][Mx] (padded index) twice
    const int row0 = blockIdx.x * G, gr = min(G, My - row0);
    double2* rows = S + ((size_t)blockIdx.y * My + row0) * Mx;
    for (int t = threadIdx.x; t < G * Mx; t += blockDim.x) sd[sx(t)] = t < gr * Mx ? rows[t] : make_double2(0, 0);
    __syncthreads();
    const double2* res = fft_smem<false>(sd, sd + padded(G * Mx), G, fx, twx);
    for (int t = threadIdx.x; t < gr * Mx; t += blockDim.x) rows[t] = res[sx(t)];
}

// forward FFT along y of G columns of one of the six fields of one mode, into Mhat [k][Mx][My][6]
// (the real part of the even fields a_ij, the imaginary part of the odd fields b_i3)
__global__ void __launch_bounds__(kSetupThreads) k_fft_dense_cols(const double2* __restrict__ S, int Mx, int My,
                                                                   Fft1D fy, int G, int k0,
                                                                   const double2* __restrict__ twy,
                                                                   double* __restrict__ mhat) {
    extern __shared__ double2 sd[];  // [G][My] (padded index) twice
    const int kk = blockIdx.y / 6, f = blockIdx.y - 6 * kk, xi0 = blockIdx.x * G, gc = min(G, Mx - xi0);
    const double2* base = S + ((size_t)kk * 6 + f) * My * Mx;
    for (int t = threadIdx.x; t < G * My; t += blockDim.x) {
        const int g = t % G, y = t / G;
        sd[sx(g * My + y)] = g < gc ? base[(size_t)y * Mx + xi0 + g] : make_double2(0, 0);
    }
    __syncthreads();
    const double2* res = fft_smem<false>(sd, sd + padded(G * My), G, fy, twy);
    for (int t = threadIdx.x; t < gc * My; t += blockDim.x) {
        const int et = t % My, g = t / My;
        const double2 v = res[sx(g * My + et)];
        mhat[(((size_t)(k0 + kk) * Mx + xi0 + g) * My + et) * 6 + f] = f < 4 ? v.x : v.y;
    }
}

}  // namespace

void fft_free(Plan& P) {
    FftGrid* F = P.fft;
    if (!F) return;
    void* bufs[] = {F->d_row_i, F->d_ent_i,  F->d_row_p, F->d_ent_p,   F->d_ypos_i,  F->d_ypos_p, F->d_twx,
                    F->d_twy,   F->d_mhat,   F->d_T1,    F->d_T2,      F->d_used,    F->d_mirror, F->d_mhat32,
                    F->d_twx32, F->d_twy32};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete F;
    P.fft = nullptr;
}

void fft_info(const Plan& P, int* mx, int* my, int* rows_i, int* rows_p, int* chunk_items) {
    const FftGrid* F = P.fft;
    *mx = F ? F->Mx : 0, *my = F ? F->My : 0;
    *rows_i = F ? F->ny_i : 0, *rows_p = F ? F->ny_p : 0;
    *chunk_items = F ? F->Q : 0;
}

// the FP32 copies of the transformed kernel and the twiddles (FBC_PREC_FFT32), once
static int fft_prepare32(Plan& P) {
    FftGrid* F = P.fft;
    if (F->d_mhat32) return FBC_OK;
    const size_t n = (size_t)P.K * F->Mx * F->My * 6;
    std::vector<float2> twx(F->Mx), twy(F->My);
    for (int j = 0; j < F->Mx; j++)
        twx[j] = make_float2((float)cos(2.0 * M_PI * j / F->Mx), (float)-sin(2.0 * M_PI * j / F->Mx));
    for (int j = 0; j < F->My; j++)
        twy[j] = make_float2((float)cos(2.0 * M_PI * j / F->My), (float)-sin(2.0 * M_PI * j / F->My));
    cudaError_t e = cudaMalloc((void**)&F->d_mhat32, n * sizeof(float));
    if (!e) e = cudaMalloc((void**)&F->d_twx32, twx.size() * sizeof(float2));
    if (!e) e = cudaMalloc((void**)&F->d_twy32, twy.size() * sizeof(float2));
    if (!e) e = cudaMemcpy(F->d_twx32, twx.data(), twx.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(F->d_twy32, twy.data(), twy.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e) {
        for (void* b : {(void*)F->d_mhat32, (void*)F->d_twx32, (void*)F->d_twy32})
            if (b) cudaFree(b);
        F->d_mhat32 = nullptr, F->d_twx32 = F->d_twy32 = nullptr;
        char msg[256];
        snprintf(msg, sizeof(msg), "in-plane FFT (FP32) setup: %s", cudaGetErrorString(e));
        return report_error(e == cudaErrorMemoryAllocation ? FBC_ERR_OOM : FBC_ERR_CUDA, msg);
    }
    const size_t b = n * sizeof(float) + (twx.size() + twy.size()) * sizeof(float2);
    F->bytes += b;
    P.workspace_bytes += b;
    return FBC_OK;
}

int fft_prepare(Plan& P, int precision) {
    if (P.fft) return precision == FBC_PREC_FFT32 ? fft_prepare32(P) : FBC_OK;
    char msg[256];
    // the differences that occur (device list of the plan)
    std::vector<int2> used(P.n_used);
    if (P.n_used && cudaMemcpy(used.data(), P.d_used, sizeof(int2) * P.n_used, cudaMemcpyDeviceToHost))
        return report_error(FBC_ERR_CUDA, "in-plane FFT: copy of the difference list failed");
    int ex = 0, ey = 0;
    std::set<std::pair<int, int>> uset;
    for (const int2& d : used) {
        ex = std::max(ex, std::abs(d.x)), ey = std::max(ey, std::abs(d.y));
        uset.insert({d.x, d.y});
    }
    FftGrid* F = new (std::nothrow) FftGrid();
    if (!F) return report_error(FBC_ERR_OOM, "host allocation failed");
    if (2 * ex + 1 > 2048 || 2 * ey + 1 > 2048) {
        delete F;
        snprintf(msg, sizeof(msg), "in-plane FFT: differences span %d x %d, above 2048 per side", 2 * ex + 1,
                 2 * ey + 1);
        return report_error(FBC_ERR_UNSUPPORTED, msg);
    }
    F->fx = choose_length(2 * ex + 1), F->fy = choose_length(2 * ey + 1);
    F->Mx = F->fx.N, F->My = F->fy.N;
    const int Mx = F->Mx, My = F->My;
    int ox = 1 << 30, oy = 1 << 30;
    for (int s = 0; s < P.NIpad; s++)
        if (P.perm_i[s] >= 0) ox = std::min(ox, P.xy_i_sorted[s].x), oy = std::min(oy, P.xy_i_sorted[s].y);
    auto rows_of = [&](const std::vector<int>& perm, const std::vector<int2>& xy, int npad, std::vector<int>& row,
                       std::vector<int2>& ent, std::vector<int>& ypos) -> bool {
        std::map<int, std::vector<int2>> by_y;
        for (int s = 0; s < npad; s++)
            if (perm[s] >= 0) by_y[xy[s].y].push_back(make_int2(xy[s].x, s));
        std::set<int> yres;
        row.assign(1, 0);
        for (auto& kv : by_y) {
            const int yr = (((kv.first - oy) % My) + My) % My;
            if (!yres.insert(yr).second) return false;
            std::set<int> xres;
            for (const int2& e : kv.second) {
                const int xr = (((e.x - ox) % Mx) + Mx) % Mx;
                if (!xres.insert(xr).second) return false;
                ent.push_back(make_int2(xr | ((int)ypos.size() << 12), e.y));  // row index in the upper bits
            }
            row.push_back((int)ent.size());
            ypos.push_back(yr);
        }
        return true;
    };
    std::vector<int> row_i, row_p, ypos_i, ypos_p;
    std::vector<int2> ent_i, ent_p;
    if (!rows_of(P.perm_i, P.xy_i_sorted, P.NIpad, row_i, ent_i, ypos_i) ||
        !rows_of(P.perm_p, P.xy_p_sorted, P.NPpad, row_p, ent_p, ypos_p)) {
        delete F;
        return report_error(FBC_ERR_UNSUPPORTED, "in-plane FFT: two sites share a grid residue");
    }
    F->ny_i = (int)ypos_i.size(), F->ny_p = (int)ypos_p.size();
    std::vector<unsigned char> mirror(used.size());
    for (size_t u = 0; u < used.size(); u++) mirror[u] = uset.count({-used[u].x, -used[u].y}) ? 0 : 1;
    // workspace for Q (rhs, mode) items at a time, at most about 1 GiB
    const size_t per_item = (size_t)Mx * (F->ny_i + F->ny_p) * 3 * sizeof(double2);
    const size_t items = (size_t)P.opt.max_rhs * P.K;
    F->Q = (int)std::max<size_t>(1, std::min<size_t>({items, (size_t)65535, ((size_t)1 << 30) / per_item}));
    std::vector<double2> twx(Mx), twy(My);
    for (int j = 0; j < Mx; j++) twx[j] = make_double2(cos(2.0 * M_PI * j / Mx), -sin(2.0 * M_PI * j / Mx));
    for (int j = 0; j < My; j++) twy[j] = make_double2(cos(2.0 * M_PI * j / My), -sin(2.0 * M_PI * j / My));
    cudaError_t e = cudaSuccess;
    size_t bytes = 0;
    auto alloc = [&](auto** p, size_t n) {
        if (e) return;
        e = cudaMalloc((void**)p, std::max<size_t>(1, n) * sizeof(**p));
        bytes += n * sizeof(**p);
    };
    auto up = [&](auto* dst, const auto& src) {
        if (!e && !src.empty()) e = cudaMemcpy(dst, src.data(), src.size() * sizeof(src[0]), cudaMemcpyHostToDevice);
    };
    alloc(&F->d_row_i, row_i.size());
    alloc(&F->d_ent_i, ent_i.size());
    alloc(&F->d_row_p, row_p.size());
    alloc(&F->d_ent_p, ent_p.size());
    alloc(&F->d_ypos_i, ypos_i.size());
    alloc(&F->d_ypos_p, ypos_p.size());
    alloc(&F->d_twx, twx.size());
    alloc(&F->d_twy, twy.size());
    alloc(&F->d_mhat, (size_t)P.K * Mx * My * 6);
    alloc(&F->d_T1, (size_t)F->Q * Mx * F->ny_i * 3);
    alloc(&F->d_T2, (size_t)F->Q * Mx * F->ny_p * 3);
    alloc(&F->d_used, used.size());
    alloc(&F->d_mirror, mirror.size());
    up(F->d_row_i, row_i), up(F->d_ent_i, ent_i), up(F->d_row_p, row_p), up(F->d_ent_p, ent_p);
    up(F->d_ypos_i, ypos_i), up(F->d_ypos_p, ypos_p), up(F->d_twx, twx), up(F->d_twy, twy);
    up(F->d_used, used), up(F->d_mirror, mirror);
    F->n_used = (int)used.size();
    F->bytes = bytes;
    P.fft = F;
    if (e) {
        fft_free(P);
        snprintf(msg, sizeof(msg), "in-plane FFT setup: %s", cudaGetErrorString(e));
        return report_error(e == cudaErrorMemoryAllocation ? FBC_ERR_OOM : FBC_ERR_CUDA, msg);
    }
    P.workspace_bytes += bytes;
    return precision == FBC_PREC_FFT32 ? fft_prepare32(P) : FBC_OK;
}

bool fft_ready(const Plan& P, int precision) {
    return P.fft && P.fft->d_mhat && (precision != FBC_PREC_FFT32 || P.fft->d_mhat32);
}

cudaError_t launch_fft_tables(Plan& P, int precision, cudaStream_t st) {
    FftGrid* F = P.fft;
    if (!fft_ready(P, precision)) return cudaErrorInvalidValue;
    const int Mx = F->Mx, My = F->My;
    const size_t per_k = (size_t)6 * Mx * My * sizeof(double2);
    const int nk = (int)std::max<size_t>(1, std::min<size_t>(P.K, ((size_t)512 << 20) / per_k));
    double2* S = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&S, per_k * nk, st);
    if (e) return e;
    const int Gr = std::max(1, std::min(My, kRowElems / Mx));
    const int Gc = std::max(1, std::min(Mx, kRowElems / My));
    const size_t smem_dr = (size_t)2 * padded(Gr * Mx) * sizeof(double2);
    const size_t smem_dc = (size_t)2 * padded(Gc * My) * sizeof(double2);
    if (smem_dr > 48 * 1024)
        cudaFuncSetAttribute(k_fft_dense_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dr);
    if (smem_dc > 48 * 1024)
        cudaFuncSetAttribute(k_fft_dense_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dc);
    for (int k0 = 0; k0 < P.K && !e; k0 += nk) {
        const int n = std::min(nk, P.K - k0);
        e = cudaMemsetAsync(S, 0, per_k * n, st);
        if (e) break;
        const long long threads = (long long)F->n_used * n;
        if (threads > 0) {
            k_fft_place<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(P.d_table, F->d_used, F->d_mirror,
                                                                           F->n_used, k0, n, P.Dx, P.Dy, P.box_x0,
                                                                           P.box_y0, Mx, My, S);
            if ((e = cudaGetLastError())) break;
        }
        k_fft_dense_rows<<<dim3((My + Gr - 1) / Gr, n * 6), kSetupThreads, smem_dr, st>>>(
            S, Mx, My, F->fx, Gr, F->d_twx);
        if ((e = cudaGetLastError())) break;
        k_fft_dense_cols<<<dim3((Mx + Gc - 1) / Gc, n * 6), kSetupThreads, smem_dc, st>>>(
            S, Mx, My, F->fy, Gc, k0, F->d_twy, F->d_mhat);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(S, st);
    if (!e && !e2 && precision == FBC_PREC_FFT32) {
        k_fft_to_f32<<<1216, 256, 0, st>>>(F->d_mhat, F->d_mhat32, (size_t)P.K * Mx * My * 6);
        e = cudaGetLastError();
    }
    return e ? e : e2;
}

// P1, P2, P3 over items [i_begin, i_end) in chunks of q_max items, complex type of R
template <typename R>
static cudaError_t run_fft_items(FftArgs A, const FftGrid* F, int i_begin, int i_end, int q_max, cudaStream_t st) {
    const int Gr = std::max(1, kRowElems / F->Mx);
    const int Gc = std::max(1, std::min(F->Mx, kRowElems / F->My));
    div_magic(Gr, &A.mG, &A.lG);
    div_magic(F->ny_i, &A.mNyi, &A.lNyi);
    div_magic(F->ny_p, &A.mNyp, &A.lNyp);
    div_magic(F->My, &A.mMy, &A.lMy);
    const size_t smem_r = (size_t)2 * padded(Gr * 3 * F->Mx) * sizeof(Cx<R>);  // data and scratch
    const size_t smem_c = (size_t)2 * padded(Gc * 3 * F->My) * sizeof(Cx<R>);
    if (smem_r > 48 * 1024) {
        cudaFuncSetAttribute(k_fft_rows_fwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r);
        cudaFuncSetAttribute(k_fft_rows_inv<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r);
    }
    if (smem_c > 48 * 1024)
        cudaFuncSetAttribute(k_fft_cols<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c);
    for (int i0 = i_begin; i0 < i_end; i0 += q_max) {
        const int q = std::min(q_max, i_end - i0);
        A.item0 = i0;
        k_fft_rows_fwd<R><<<dim3((F->ny_i + Gr - 1) / Gr, q), kFftThreads, smem_r, st>>>(A, Gr);
        cudaError_t e = cudaGetLastError();
        if (e) return e;
        k_fft_cols<R><<<dim3((F->Mx + Gc - 1) / Gc, q), kFftThreads, smem_c, st>>>(A, Gc);
        if ((e = cudaGetLastError())) return e;
        k_fft_rows_inv<R><<<dim3((F->ny_p + Gr - 1) / Gr, q), kFftThreads, smem_r, st>>>(A, Gr);
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_contract_fft(Plan& P, int n_rhs, cudaStream_t st) {
    FftGrid* F = P.fft;
    if (!fft_ready(P, P.precision)) return cudaErrorInvalidValue;
    FftArgs A{};
    A.fh = P.d_fh, A.uh = P.d_uh, A.T1 = F->d_T1, A.T2 = F->d_T2;
    A.row_i = F->d_row_i, A.ent_i = F->d_ent_i, A.row_p = F->d_row_p, A.ent_p = F->d_ent_p;
    A.ypos_i = F->d_ypos_i, A.ypos_p = F->d_ypos_p;
    A.fx = F->fx, A.fy = F->fy;
    A.Mx = F->Mx, A.My = F->My, A.ny_i = F->ny_i, A.ny_p = F->ny_p;
    A.R = n_rhs, A.K = P.K, A.NIpad = P.NIpad, A.NPpad = P.NPpad;
    A.scale = 1.0 / ((double)F->Mx * (double)F->My);
    const int items = n_rhs * P.K;
    // FP64: every mode; FP32 form: the logarithmic k = 0 mode (items 0 .. n_rhs - 1) stays FP64
    const int n64 = P.precision == FBC_PREC_FFT32 ? n_rhs : items;
    A.mhat = F->d_mhat, A.twx = F->d_twx, A.twy = F->d_twy;
    cudaError_t e = run_fft_items<double>(A, F, 0, n64, F->Q, st);
    if (e || n64 == items) return e;
    A.mhat = F->d_mhat32, A.twx = F->d_twx32, A.twy = F->d_twy32;
    return run_fft_items<float>(A, F, n64, items, std::min(2 * F->Q, 65535), st);
}

}  // namespace fbc

// ---- lattice Green function near field (App.) ------------------------------------------------------
//
// The lattice Green function of a harmonic block stencil K_h is the inverse transform of its inverted
// Fourier symbol; in mode k of the line-periodic lattice
//     g^k(d) = (2 pi)^-2 int D(theta_x, theta_y, 2 pi k / L)^-1 exp(i theta . d),
//     D(theta) = sum_n K(n) exp(-i theta . n) = sum_n K(n) cos(theta . n)   (K(-n) = K(n)).
// On an n x n zone grid the trapezoid rule is an inverse DFT: the six fields of D^-1, placed at -theta,
// go through the forward 2D transform above, and g^k(d) is read at d mod n.  The k = 0 mode is
// singular at theta = 0 (left out: the zero-mean function) and is defined only up to a constant, so
// it is shifted by the blending constant C = g_lat^0(d_ref) - g_cont^0(d_ref) at a reference
// difference beyond the cut-off (App.); a constant in real space only touches k = 0.

namespace fbc {
namespace {

// S [nk][6][n][n]: fields A11 A12 A22 A33 B13 B23 of D^-1 at theta = (-2 pi x / n, -2 pi y / n, 2 pi k / L)
__global__ void k_zone_fill(const double* __restrict__ Kb, unsigned mask, int L, int k0, int nk, int n,
                            double2* __restrict__ S) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nk * n * n) return;
    const int x = (int)(t % n);
    const long long rem = t / n;
    const int y = (int)(rem % n), kk = (int)(rem / n), k = k0 + kk;
    const double tx = -2.0 * M_PI * x / n, ty = -2.0 * M_PI * y / n, tz = 2.0 * M_PI * k / L;
    double D[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = 0; j < 27; j++) {
        if (!((mask >> j) & 1u)) continue;
        const int nx = j / 9 - 1, ny = (j / 3) % 3 - 1, nz = j % 3 - 1;
        const double cs = cos(tx * nx + ty * ny + tz * nz);
        for (int e = 0; e < 9; e++) D[e] = fma(Kb[9 * j + e], cs, D[e]);
    }
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (!(k == 0 && x == 0 && y == 0)) {
        // symmetric 3x3 inverse by cofactors
        const double a = D[0], b = D[1], c = D[2], e = D[4], f = D[5], i = D[8];
        const double c00 = e * i - f * f, c01 = c * f - b * i, c02 = b * f - c * e;
        const double det = a * c00 + b * c01 + c * c02;
        const double r = 1.0 / det;
        v[0] = c00 * r;                    // (1,1)
        v[1] = c01 * r;                    // (1,2)
        v[2] = (a * i - c * c) * r;        // (2,2)
        v[3] = (a * e - b * b) * r;        // (3,3)
        v[4] = c02 * r;                    // (1,3)
        v[5] = (b * c - a * f) * r;        // (2,3)
    }
    double2* base = S + (size_t)kk * 6 * n * n + (size_t)y * n + x;
    for (int fld = 0; fld < 6; fld++) base[(size_t)fld * n * n] = make_double2(v[fld], 0.0);
}

// table entries of the near differences for modes k0 .. k0 + nk - 1 from the transformed fields
// Z [nk][n][n][6] (scaled by 1 / n^2); k = 0 minus the blending constant
__global__ void k_zone_extract(const double* __restrict__ Z, int n, int k0, int nk, const int2* __restrict__ near_d,
                               const int* __restrict__ near_idx, int n_near, int2 dref, int ref_idx, double* tab,
                               size_t slice) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nk * n_near * 6) return;
    const int f = t % 6, e = (t / 6) % n_near, kk = t / (6 * n_near), k = k0 + kk;
    const double s = 1.0 / ((double)n * (double)n);
    auto at = [&](int2 d) {
        const int px = ((d.x % n) + n) % n, py = ((d.y % n) + n) % n;
        return Z[(((size_t)kk * n + px) * n + py) * 6 + f] * s;
    };
    double v = at(near_d[e]);
    if (k == 0 && ref_idx >= 0) v -= at(dref) - tab[(size_t)ref_idx * 6 + f];
    tab[((size_t)k * slice + near_idx[e]) * 6 + f] = v;
}

}  // namespace
}  // namespace fbc

extern "C" int fbc_plan_lattice_near_field(fbc_plan* plan, const double* K, double r_cut, int32_t ref_dx,
                                           int32_t ref_dy, int32_t n_zone) {
    using namespace fbc;
    report_error(FBC_OK, "");
    char msg[256];
    if (!plan || !K) return report_error(FBC_ERR_INVALID_ARG, "plan or K is NULL");
    Plan& P = plan->p;
    if (P.host_only) return report_error(FBC_ERR_INVALID_ARG, "host-only plan");
    if (!P.tabulated) return report_error(FBC_ERR_NOT_TABULATED, "tabulate the plan first");
    if (P.sur || P.tables_released || !P.d_table)
        return report_error(FBC_ERR_UNSUPPORTED, "the plan serves a surrogate; detach it first");
    if (!(r_cut > 0.0) || !std::isfinite(r_cut)) return report_error(FBC_ERR_INVALID_ARG, "need r_cut > 0");
    const bool blend = ref_dx != 0 || ref_dy != 0;
    if (blend && (double)ref_dx * ref_dx + (double)ref_dy * ref_dy <= r_cut * r_cut)
        return report_error(FBC_ERR_INVALID_ARG, "the reference difference must lie beyond r_cut");
    if (n_zone < 16 || n_zone > 2048) return report_error(FBC_ERR_INVALID_ARG, "n_zone must be in [16, 2048]");
    // the stencil: finite, K(-n) = K(n), symmetric blocks K(n) = K(n)^T (with K(-n) = K(n) this makes the
    // symbol real and symmetric, which the cofactor inverse of k_zone_fill assumes: it reads one triangle),
    // and mirror-symmetric in the line direction (the six-real layout)
    unsigned mask = 0;
    for (int j = 0; j < 27; j++) {
        const int nx = j / 9 - 1, ny = (j / 3) % 3 - 1, nz = j % 3 - 1;
        const int jm = (1 - nx) * 9 + (1 - ny) * 3 + (1 - nz), jz = (nx + 1) * 9 + (ny + 1) * 3 + (1 - nz);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                const double v = K[9 * j + 3 * a + b];
                if (!std::isfinite(v)) return report_error(FBC_ERR_INVALID_ARG, "K has a non-finite entry");
                if (v != 0.0) mask |= 1u << j;
                if (std::fabs(v - K[9 * jm + 3 * a + b]) > 1e-14 * (1.0 + std::fabs(v)))
                    return report_error(FBC_ERR_UNSUPPORTED, "the stencil must satisfy K(-n) = K(n)");
                if (std::fabs(v - K[9 * j + 3 * b + a]) > 1e-14 * (1.0 + std::fabs(v)))
                    return report_error(FBC_ERR_UNSUPPORTED, "the stencil blocks must be symmetric, K(n) = K(n)^T");
                const double sg = ((a == 2) != (b == 2)) ? -1.0 : 1.0;  // M K M with M = diag(1, 1, -1)
                if (std::fabs(v - sg * K[9 * jz + 3 * a + b]) > 1e-14 * (1.0 + std::fabs(v)))
                    return report_error(FBC_ERR_UNSUPPORTED, "the stencil must be mirror-symmetric along the line");
            }
    }
    // near differences from the plan's difference list; the reference must be one of its differences
    std::vector<int2> used(P.n_used);
    if (P.n_used && cudaMemcpy(used.data(), P.d_used, sizeof(int2) * P.n_used, cudaMemcpyDeviceToHost))
        return report_error(FBC_ERR_CUDA, "copy of the difference list failed");
    std::vector<int2> near_d;
    std::vector<int> near_idx;
    const int2 dref = make_int2(ref_dx, ref_dy);
    bool ref_found = false;
    int dmax = 0;
    for (const int2& d : used) {
        if ((double)d.x * d.x + (double)d.y * d.y <= r_cut * r_cut) {
            near_d.push_back(d);
            near_idx.push_back((d.y - P.box_y0) * P.Dx + (d.x - P.box_x0));
            dmax = std::max(dmax, std::max(std::abs(d.x), std::abs(d.y)));
        }
        ref_found = ref_found || (d.x == dref.x && d.y == dref.y);
    }
    if (blend && !ref_found)
        return report_error(FBC_ERR_INVALID_ARG, "the reference difference is not in the plan's table");
    if (near_d.empty()) {  // nothing within the cut-off
        P.opt.flags |= kPlanNearFieldSet;
        return FBC_OK;
    }
    const int ref_idx = blend ? (dref.y - P.box_y0) * P.Dx + (dref.x - P.box_x0) : -1;
    dmax = std::max(dmax, std::max(std::abs(dref.x), std::abs(dref.y)));
    const Fft1D fz = choose_length(n_zone);
    const int n = fz.N;
    if (n < 2 * dmax + 2) {
        snprintf(msg, sizeof(msg), "zone grid %d too small for differences up to %d", n, dmax);
        return report_error(FBC_ERR_INVALID_ARG, msg);
    }
    std::vector<double2> tw(n);
    for (int j = 0; j < n; j++) tw[j] = make_double2(cos(2.0 * M_PI * j / n), -sin(2.0 * M_PI * j / n));
    const size_t per_k = (size_t)n * n * (6 * sizeof(double2) + 6 * sizeof(double));
    const int nk = (int)std::max<size_t>(1, std::min<size_t>(P.K, ((size_t)512 << 20) / per_k));
    double* dK = nullptr;
    double2* dtw = nullptr;
    double2* S = nullptr;
    double* Z = nullptr;
    int2* dnd = nullptr;
    int* dni = nullptr;
    cudaError_t e = cudaMalloc((void**)&dK, 27 * 9 * sizeof(double));
    if (!e) e = cudaMalloc((void**)&dtw, n * sizeof(double2));
    if (!e) e = cudaMalloc((void**)&S, (size_t)nk * 6 * n * n * sizeof(double2));
    if (!e) e = cudaMalloc((void**)&Z, (size_t)nk * n * n * 6 * sizeof(double));
    if (!e) e = cudaMalloc((void**)&dnd, near_d.size() * sizeof(int2));
    if (!e) e = cudaMalloc((void**)&dni, near_idx.size() * sizeof(int));
    if (!e) e = cudaMemcpy(dK, K, 27 * 9 * sizeof(double), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(dtw, tw.data(), n * sizeof(double2), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(dnd, near_d.data(), near_d.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(dni, near_idx.data(), near_idx.size() * sizeof(int), cudaMemcpyHostToDevice);
    const int Gr = std::max(1, std::min(n, kRowElems / n));
    const size_t smem = (size_t)2 * padded(Gr * n) * sizeof(double2);
    if (!e && smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_fft_dense_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (!e) e = cudaFuncSetAttribute(k_fft_dense_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    const size_t slice = (size_t)P.Dy * P.Dx;
    for (int k0 = 0; k0 < P.K && !e; k0 += nk) {
        const int m = std::min(nk, P.K - k0);
        const long long pts = (long long)m * n * n;
        k_zone_fill<<<(unsigned)((pts + 255) / 256), 256>>>(dK, mask, P.L, k0, m, n, S);
        if ((e = cudaGetLastError())) break;
        k_fft_dense_rows<<<dim3((n + Gr - 1) / Gr, m * 6), kSetupThreads, smem>>>(S, n, n, fz, Gr, dtw);
        if ((e = cudaGetLastError())) break;
        k_fft_dense_cols<<<dim3((n + Gr - 1) / Gr, m * 6), kSetupThreads, smem>>>(S, n, n, fz, Gr, 0, dtw, Z);
        if ((e = cudaGetLastError())) break;
        const int work = m * (int)near_d.size() * 6;
        k_zone_extract<<<(work + 255) / 256, 256>>>(Z, n, k0, m, dnd, dni, (int)near_d.size(), dref, ref_idx,
                                                    P.d_table, slice);
        e = cudaGetLastError();
    }
    if (!e) e = cudaDeviceSynchronize();
    for (void* b : {(void*)dK, (void*)dtw, (void*)S, (void*)Z, (void*)dnd, (void*)dni})
        if (b) cudaFree(b);
    if (!e && P.precision != FBC_PREC_FP64) {
        e = launch_derive_tables(P, P.precision, 0);
        if (!e) e = cudaDeviceSynchronize();
    }
    if (e) {
        snprintf(msg, sizeof(msg), "lattice near field: %s", cudaGetErrorString(e));
        return report_error(e == cudaErrorMemoryAllocation ? FBC_ERR_OOM : FBC_ERR_CUDA, msg);
    }
    P.opt.flags |= kPlanNearFieldSet;
    return FBC_OK;
}
