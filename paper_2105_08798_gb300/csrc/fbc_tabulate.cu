// Kernel-table generation (setup, FP64).
//
// Stage 1 (periodic kernel): for every in-plane difference d that occurs and
// every repeat offset s in [0, L/2], the regularised image sum of Sec. 3.1
// (Eqs. 32, 35) extrapolated with Richardson's formula (Eq. 36):
//     G~(d, s) = G_n + sum_{m=n+1}^{n+N} W_m t_m,
//     G_n = G(d, s c) + sum_{m=1}^{n} t_m,
//     t_m = G(d, s c + m l3) + G(d, s c - m l3) - G(0, 0, m l3) - G(0, 0, -m l3),
// with W_m the cumulative weights computed on the host (algebraically the same
// as Eq. 36, arranged so that the large alternating weights only multiply the
// small increments t_m).  At s = L/2 the two centred representatives
// +-L/2 are averaged, which for a mirror-symmetric medium keeps the even
// entries and zeroes the odd ones.
//
// Stage 2 (line DFT): g^k(d) = sum_s G~(d, s) exp(-2 pi i k s / L) for
// k = 0..L/2.  With the mirror symmetry G~(d, L - s) = M G~(d, s) M,
// M = diag(1, 1, -1), the even entries give a cosine sum (real part) and the
// odd entries a sine sum (imaginary part):
//     A(k) = G(0) + (-1)^k G(L/2) + 2 sum_{s=1}^{L/2-1} G(s) cos(2 pi k s / L),
//     B(k) = -2 sum_{s=1}^{L/2-1} G(s) sin(2 pi k s / L).
//
// The continuum Green function (Eq. 33) is Kelvin's closed form for an
// isotropic medium and Barnett's integral over the unit circle normal to r,
//     G(r) = 1/(8 pi^2 |r|) int_0^{2 pi} (zz)^{-1} dpsi,
// for a cubic one, evaluated by the trapezoid rule on [0, pi) (the integrand
// has period pi) with the nodes' cosines and sines in constant memory.
#include <cmath>
#include <vector>

#include "fbc_internal.cuh"

namespace fbc {
namespace {

__constant__ MaterialDev c_mat;
__constant__ TabulateParams c_tp;
__constant__ double c_qcos[kMaxQuad];
__constant__ double c_qsin[kMaxQuad];

// G as six entries (11, 12, 22, 33, 13, 23) of the symmetric tensor.
__device__ void green6(double rx, double ry, double rz, double g[6]) {
    const double R2 = rx * rx + ry * ry + rz * rz;
    const double R = sqrt(R2);
    if (c_mat.kind == FBC_MATERIAL_ISOTROPIC) {
        const double pre = c_mat.kelvin_pre / R;
        const double iR2 = 1.0 / R2;
        const double a = c_mat.kelvin_a;
        g[0] = pre * (a + rx * rx * iR2);
        g[1] = pre * (rx * ry * iR2);
        g[2] = pre * (a + ry * ry * iR2);
        g[3] = pre * (a + rz * rz * iR2);
        g[4] = pre * (rx * rz * iR2);
        g[5] = pre * (ry * rz * iR2);
        return;
    }
    // unit direction and an orthonormal pair spanning the plane normal to it
    const double iR = 1.0 / R;
    const double hx = rx * iR, hy = ry * iR, hz = rz * iR;
    double e1x, e1y, e1z;
    const double rho2 = hx * hx + hy * hy;
    if (rho2 > 1e-24) {
        const double ir = rsqrt(rho2);
        e1x = -hy * ir, e1y = hx * ir, e1z = 0.0;
    } else {
        e1x = 1.0, e1y = 0.0, e1z = 0.0;
    }
    const double e2x = hy * e1z - hz * e1y;
    const double e2y = hz * e1x - hx * e1z;
    const double e2z = hx * e1y - hy * e1x;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;  // 11 22 33 23 13 12
    const int nq = c_mat.nquad;
    for (int q = 0; q < nq; q++) {
        const double cq = c_qcos[q], sq = c_qsin[q];
        const double zx = cq * e1x + sq * e2x;
        const double zy = cq * e1y + sq * e2y;
        const double zz = cq * e1z + sq * e2z;
        const double p[6] = {zx * zx, zy * zy, zz * zz, zy * zz, zx * zz, zx * zy};
        double m[6];
#pragma unroll
        for (int I = 0; I < 6; I++) {
            double v = 0.0;
#pragma unroll
            for (int J = 0; J < 6; J++) v = fma(c_mat.K[6 * I + J], p[J], v);
            m[I] = v;
        }
        // symmetric 3x3 inverse by the adjugate; m = (a, b, c, d, e, f) = (00, 11, 22, 12, 02, 01)
        const double a = m[0], b = m[1], c = m[2], d = m[3], e = m[4], f = m[5];
        const double A00 = b * c - d * d, A11 = a * c - e * e, A22 = a * b - f * f;
        const double A12 = e * f - a * d, A02 = d * f - b * e, A01 = d * e - c * f;
        const double idet = 1.0 / (a * A00 + f * A01 + e * A02);
        s0 = fma(A00, idet, s0);
        s1 = fma(A11, idet, s1);
        s2 = fma(A22, idet, s2);
        s3 = fma(A12, idet, s3);
        s4 = fma(A02, idet, s4);
        s5 = fma(A01, idet, s5);
    }
    // 2 * (pi / nq) / (8 pi^2 R) = 1 / (4 pi nq R)
    const double pre = 1.0 / (4.0 * M_PI * (double)nq * R);
    g[0] = pre * s0;
    g[1] = pre * s5;
    g[2] = pre * s1;
    g[3] = pre * s2;
    g[4] = pre * s4;
    g[5] = pre * s3;
}

// Stage 1: one thread per (used difference, s in [0, L/2]).
__global__ void k_periodic(const int2* __restrict__ used, int n_used, double* __restrict__ gs) {
    const int Lh = c_tp.Lh;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)n_used * (Lh + 1);
    if (tid >= total) return;
    const int di = (int)(tid / (Lh + 1));
    const int s = (int)(tid % (Lh + 1));
    const int2 d = used[di];
    if (d.x == 0 && d.y == 0) {  // self-terms (FBC_PLAN_SELF_TERMS): filled by the lattice near field
        double* o0 = gs + ((size_t)di * (Lh + 1) + s) * 6;
        for (int t = 0; t < 6; t++) o0[t] = 0.0;
        return;
    }
    const double rx = (double)d.x, ry = (double)d.y;
    const double l3 = (double)c_tp.L * c_tp.c;
    const double z0 = (double)s * c_tp.c;  // centred representative: s <= L/2
    double acc[6], g[6], h[6], gr[6], hr[6];
    green6(rx, ry, z0, acc);
    const int n = c_tp.rich_n, N = c_tp.rich_N;
    double tail[6] = {0, 0, 0, 0, 0, 0};
    for (int m = 1; m <= n + N; m++) {
        const double zm = (double)m * l3;
        green6(rx, ry, z0 + zm, g);
        green6(rx, ry, z0 - zm, h);
        green6(0.0, 0.0, zm, gr);
        green6(0.0, 0.0, -zm, hr);
        if (m <= n) {
#pragma unroll
            for (int t = 0; t < 6; t++) acc[t] += ((g[t] + h[t]) - (gr[t] + hr[t]));
        } else {
            const double w = c_tp.W[m - n - 1];
#pragma unroll
            for (int t = 0; t < 6; t++) tail[t] = fma(w, (g[t] + h[t]) - (gr[t] + hr[t]), tail[t]);
        }
    }
    double* o = gs + ((size_t)di * (Lh + 1) + s) * 6;
#pragma unroll
    for (int t = 0; t < 6; t++) o[t] = acc[t] + tail[t];
    if (s == Lh) {  // average of +L/2 and -L/2: odd entries cancel
        o[4] = 0.0;
        o[5] = 0.0;
    }
    if (s == 0) {  // exactly odd in s: zero at s = 0
        o[4] = 0.0;
        o[5] = 0.0;
    }
}

// Stage 2: one CTA per used difference; threads over k.
__global__ void k_line_dft(const int2* __restrict__ used, const double* __restrict__ gs,
                           const double2* __restrict__ twL, double* __restrict__ table) {
    extern __shared__ double sg[];  // [Lh+1][6]
    const int Lh = c_tp.Lh, L = c_tp.L, K = c_tp.K;
    const int di = blockIdx.x;
    const double* src = gs + (size_t)di * (Lh + 1) * 6;
    for (int t = threadIdx.x; t < (Lh + 1) * 6; t += blockDim.x) sg[t] = src[t];
    __syncthreads();
    const int2 d = used[di];
    const int ix = d.x - c_tp.box_x0, iy = d.y - c_tp.box_y0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double sgn = (k & 1) ? -1.0 : 1.0;
        double A0 = 0, A1 = 0, A2 = 0, A3 = 0, B4 = 0, B5 = 0;
        int ks = 0;
        for (int s = 1; s < Lh; s++) {
            ks += k;
            if (ks >= L) ks -= L;
            const double2 cs = twL[ks];
            const double* gp = sg + s * 6;
            A0 = fma(gp[0], cs.x, A0);
            A1 = fma(gp[1], cs.x, A1);
            A2 = fma(gp[2], cs.x, A2);
            A3 = fma(gp[3], cs.x, A3);
            B4 = fma(gp[4], cs.y, B4);
            B5 = fma(gp[5], cs.y, B5);
        }
        const double* g0 = sg;
        const double* gh = sg + Lh * 6;
        double* o = table + (((size_t)k * c_tp.Dy + iy) * c_tp.Dx + ix) * 6;
        o[0] = g0[0] + sgn * gh[0] + 2.0 * A0;
        o[1] = g0[1] + sgn * gh[1] + 2.0 * A1;
        o[2] = g0[2] + sgn * gh[2] + 2.0 * A2;
        o[3] = g0[3] + sgn * gh[3] + 2.0 * A3;
        o[4] = -2.0 * B4;
        o[5] = -2.0 * B5;
    }
}

// Derived tables for the reduced-precision contractions.
__global__ void k_derive_fp32(const double* __restrict__ t64, float* __restrict__ t32, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) t32[i] = (float)t64[i];
}

// Double-float split: v = hi + lo with hi = fl32(v), lo = fl32(v - hi).  Stored
// per entry as the pairs (hi0, lo0, hi1, lo1, ..., hi5, lo5): three 16-byte
// records, the layout the contraction keeps in shared memory, so that a tile's
// sub-box is one tensor copy.
__global__ void k_derive_x2(const double* __restrict__ t64, float* __restrict__ tx2, size_t n_entries) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; e < n_entries; e += stride) {
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const double v = t64[e * 6 + c];
            const float hi = (float)v;
            const float lo = (float)(v - (double)hi);
            tx2[e * 12 + 2 * c] = hi;
            tx2[e * 12 + 2 * c + 1] = lo;
        }
    }
}

}  // namespace

// The plan's medium and tabulation parameters into this file's constant memory (shared by every
// plan: uploaded again before each use).
static cudaError_t upload_tabulate_constants(Plan& P, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemcpyToSymbolAsync(c_mat, &P.mat, sizeof(MaterialDev), 0, cudaMemcpyHostToDevice, st))) return e;
    if ((e = cudaMemcpyToSymbolAsync(c_tp, &P.tp, sizeof(TabulateParams), 0, cudaMemcpyHostToDevice, st))) return e;
    if (P.mat.kind == FBC_MATERIAL_CUBIC) {
        static thread_local std::vector<double> qc, qs;
        qc.assign(kMaxQuad, 0.0);
        qs.assign(kMaxQuad, 0.0);
        for (int q = 0; q < P.mat.nquad; q++) {
            const double psi = M_PI * (double)q / (double)P.mat.nquad;
            qc[q] = cos(psi);
            qs[q] = sin(psi);
        }
        if ((e = cudaMemcpyToSymbolAsync(c_qcos, qc.data(), sizeof(double) * kMaxQuad, 0, cudaMemcpyHostToDevice, st)))
            return e;
        if ((e = cudaMemcpyToSymbolAsync(c_qsin, qs.data(), sizeof(double) * kMaxQuad, 0, cudaMemcpyHostToDevice, st)))
            return e;
        // the host vectors must outlive the asynchronous copies
        if ((e = cudaStreamSynchronize(st))) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_tabulate(Plan& P, cudaStream_t st) {
    cudaError_t e;
    if ((e = upload_tabulate_constants(P, st))) return e;
    if (P.n_used == 0) return cudaSuccess;
    const int Lh = P.L / 2;
    // process the differences in chunks so the stage-1 buffer stays bounded
    const size_t per_d = (size_t)(Lh + 1) * 6 * sizeof(double);
    int chunk = (int)std::min<size_t>((size_t)P.n_used, std::max<size_t>(1, (size_t)256 << 20) / per_d);
    if (chunk < 1) chunk = 1;
    double* gs = nullptr;
    if ((e = cudaMallocAsync((void**)&gs, per_d * chunk, st))) return e;
    const size_t smem = per_d;
    if (smem > 32 * 1024) {
        if ((e = cudaFuncSetAttribute(k_line_dft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) {
            cudaFreeAsync(gs, st);
            return e;
        }
    }
    for (int d0 = 0; d0 < P.n_used; d0 += chunk) {
        const int nd = std::min(chunk, P.n_used - d0);
        const long long threads = (long long)nd * (Lh + 1);
        const int bs = 128;
        k_periodic<<<(unsigned)((threads + bs - 1) / bs), bs, 0, st>>>(P.d_used + d0, nd, gs);
        if ((e = cudaGetLastError())) break;
        const int bt = std::min(256, std::max(32, ((P.K + 31) / 32) * 32));
        k_line_dft<<<nd, bt, smem, st>>>(P.d_used + d0, gs, P.d_twL, P.d_table);
        if ((e = cudaGetLastError())) break;
    }
    cudaError_t e2 = cudaFreeAsync(gs, st);
    return e ? e : e2;
}

// Stage-1 output of a chunk of used differences, rounded to FP32 and placed at each difference's
// cell of the box: out[cell][s][6] for s = 0..L/2.
__global__ void k_real_space_scatter(const int2* __restrict__ used, int n_used, const double* __restrict__ gs,
                                     float* __restrict__ out) {
    const int Lh = c_tp.Lh;
    const long long per = (long long)(Lh + 1) * 6;
    const long long total = (long long)n_used * per;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int di = (int)(t / per);
        const long long r = t - (long long)di * per;
        const int2 d = used[di];
        const long long cell = (long long)(d.y - c_tp.box_y0) * c_tp.Dx + (d.x - c_tp.box_x0);
        out[cell * per + r] = (float)gs[t];
    }
}

cudaError_t launch_real_space_table(Plan& P, float* out, cudaStream_t st) {
    cudaError_t e;
    if ((e = upload_tabulate_constants(P, st))) return e;
    const int Lh = P.L / 2;
    const size_t cells = (size_t)P.Dx * P.Dy;
    if ((e = cudaMemsetAsync(out, 0, cells * (Lh + 1) * 6 * sizeof(float), st))) return e;
    if (P.n_used == 0) return cudaSuccess;
    const size_t per_d = (size_t)(Lh + 1) * 6 * sizeof(double);
    int chunk = (int)std::min<size_t>((size_t)P.n_used, std::max<size_t>(1, (size_t)256 << 20) / per_d);
    if (chunk < 1) chunk = 1;
    double* gs = nullptr;
    if ((e = cudaMallocAsync((void**)&gs, per_d * chunk, st))) return e;
    for (int d0 = 0; d0 < P.n_used; d0 += chunk) {
        const int nd = std::min(chunk, P.n_used - d0);
        const long long threads = (long long)nd * (Lh + 1);
        k_periodic<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(P.d_used + d0, nd, gs);
        if ((e = cudaGetLastError())) break;
        k_real_space_scatter<<<1216, 256, 0, st>>>(P.d_used + d0, nd, gs, out);
        if ((e = cudaGetLastError())) break;
    }
    cudaError_t e2 = cudaFreeAsync(gs, st);
    return e ? e : e2;
}

cudaError_t launch_derive_tables(Plan& P, int precision, cudaStream_t st) {
    const size_t cells = (size_t)P.K * P.Dy * P.Dx;
    if (precision == FBC_PREC_FP32 || is_tensor_precision(precision)) {
        if (!P.d_table32 || !P.d_table_x2_k0) return cudaErrorInvalidValue;
        k_derive_fp32<<<1216, 256, 0, st>>>(P.d_table, P.d_table32, cells * 6);
        cudaError_t e = cudaGetLastError();
        if (e) return e;
        k_derive_x2<<<1216, 256, 0, st>>>(P.d_table, P.d_table_x2_k0, (size_t)P.Dy * P.Dx);  // k = 0 slice
        return cudaGetLastError();
    }
    if (is_fft_precision(precision)) return launch_fft_tables(P, precision, st);
    if (precision == FBC_PREC_F32X2 || precision == FBC_PREC_BF16X6) {
        if (!P.d_table_x2) return cudaErrorInvalidValue;
        k_derive_x2<<<1216, 256, 0, st>>>(P.d_table, P.d_table_x2, cells);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace fbc
