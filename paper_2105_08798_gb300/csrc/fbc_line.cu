// Transforms along the periodic line (FP64, HBM-bound).
//
// Forward (before the contraction): for each interface column b the three
// real force sequences f_c(b, q), q = 0..L-1, are transformed to
//     F_c(b, k) = sum_q f_c(b, q) exp(-2 pi i k q / L),  k = 0..L/2,
// and stored as six-vectors (Re F1, Re F2, Im F3, Im F1, Im F2, -Re F3) in
// tile-sorted column order.  Two real sequences share one complex FFT:
// z = f1 + i f2 per column, and w = f3(b) + i f3(b+1) per column pair.
// Removing the net force (a constant over all N_I L atoms) only changes the
// k = 0 mode, by -L * mean, which the projection kernel applies.
//
// Inverse (after the contraction): the contracted six-vectors give
// U_c(a, k) for k = 0..L/2; the Hermitian extension U(L - k) = conj U(k)
// makes the inverse transform real, and
//     u(a, p) <- beta u(a, p) + (alpha / L) sum_k U(a, k) exp(+2 pi i k p / L).
// Imaginary parts at k = 0 and k = L/2 are dropped (they vanish for a real
// result), as a real inverse DFT does.  The optional zero-mean step
// (Sec. 2.3.2, Eq. 23) subtracts the per-component mean over all pad atoms.
//
// The FFT is an in-place radix-2 decimation-in-time transform in shared
// memory (bit-reversed load, log2 L butterfly stages).  A CTA holds NC
// columns, i.e. 1.5 NC complex sequences of length L.
//
// Two arithmetic forms.  FP64 throughout for the FP64 and double-float
// contractions.  For the FP32 and tensor-core contractions (whose own error
// is 3e-6 or more) the FFT runs in FP32, which on GB300 is about 30x the
// FP64 rate, while the k = 0 mode stays FP64: the forward k = 0 entries are
// FP64 column sums, and the inverse adds the k = 0 term (a constant along the
// line) in FP64 after an FP32 transform of the k >= 1 modes.
#include "fbc_fft.cuh"
#include "fbc_internal.cuh"

namespace fbc {
namespace {

template <typename R>
struct Cx;
template <>
struct Cx<double> {
    using T = double2;
    __device__ static T make(double x, double y) { return make_double2(x, y); }
};
template <>
struct Cx<float> {
    using T = float2;
    __device__ static T make(float x, float y) { return make_float2(x, y); }
};

// GB300's FP64 pipe runs at about 1/64 of the FP32 rate, and conversions
// between double and float issue there too.  The FP32 forms therefore convert
// with integer bit arithmetic (d2f_int, f2d_int) and keep one FP64 add per
// output element (the k = 0 term).
// (sh, sl) += v with an exact two-sum (double-float accumulation on the FP32 pipes)
__device__ __forceinline__ void df_acc(float v, float& sh, float& sl) {
    const float t = __fadd_rn(sh, v);
    const float bb = __fsub_rn(t, sh);
    sl = __fadd_rn(sl, __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(v, bb)));
    sh = t;
}

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    T2 r;
    r.x = fma(a.x, b.x, -a.y * b.y);
    r.y = fma(a.x, b.y, a.y * b.x);
    return r;
}

__device__ __forceinline__ int bitrev(int x, int logL) { return (int)(__brev((unsigned)x) >> (32 - logL)); }

// nseq sequences of length L in buf; tw[t] = exp(-2 pi i t / L) (FP32 form: the float
// copy tw32[t] stored after the L/2 double entries); inverse uses conj.
template <typename R>
__device__ void fft_block(typename Cx<R>::T* buf, int nseq, int L, int logL, const double2* __restrict__ tw,
                          bool inverse) {
    using T2 = typename Cx<R>::T;
    const int half = L >> 1;
    for (int lh = 0; lh < logL; lh++) {
        const int h = 1 << lh;
        const int stride_tw = half >> lh;  // L / (2h)
        for (int t = threadIdx.x; t < nseq * half; t += blockDim.x) {
            const int sq = t >> (logL - 1);
            const int j = t & (half - 1);
            const int pos = j & (h - 1);
            const int grp = j >> lh;
            const int i0 = (grp << (lh + 1)) + pos;
            const int i1 = i0 + h;
            T2 w;
            if constexpr (sizeof(R) == 4) {
                // the float copy after the L/2 double entries (no conversion on the FP64 pipe)
                w = __ldg(&((const float2*)(tw + half))[pos * stride_tw]);
            } else {
                w = __ldg(&tw[pos * stride_tw]);
            }
            if (inverse) w.y = -w.y;
            T2* s = buf + (size_t)sq * L;
            const T2 a = s[i0];
            const T2 bw = cmul(s[i1], w);
            s[i0] = Cx<R>::make(a.x + bw.x, a.y + bw.y);
            s[i1] = Cx<R>::make(a.x - bw.x, a.y - bw.y);
        }
        __syncthreads();
    }
}

// Forward transform of NC columns (block blk of right-hand side r).
template <typename R>
__device__ __forceinline__ void fwd_block(const double* __restrict__ f, const int* __restrict__ perm,
                                          const double2* __restrict__ tw, double* __restrict__ fh, int n_i, int L,
                                          int logL, int K, int NIpad, int NC, int blk, int r, void* sraw) {
    using T2 = typename Cx<R>::T;
    constexpr bool kF32 = sizeof(R) == 4;
    const int logNC = __ffs(NC) - 1;  // NC and L are powers of two: shifts, no integer division
    // sbuf: [NC + NC/2][L], z sequences then w sequences
    const int b0 = blk * NC;
    T2* zs = (T2*)sraw;
    T2* ws = zs + (size_t)NC * L;
    __shared__ double s0[kF32 ? 64 : 1][3];  // FP64 column sums = the k = 0 mode (FP32 form)
    // load: each column's L x 3 block is contiguous in f
    for (int t = threadIdx.x; t < NC * L; t += blockDim.x) {
        const int j = t >> logL, q = t & (L - 1);
        const int ob = perm[b0 + j];
        const int qr = bitrev(q, logL);
        R* wp = (R*)&ws[(size_t)(j >> 1) * L + qr];
        if constexpr (kF32) {
            long long b1 = 0, b2 = 0, b3 = 0;  // raw FP64 words: nothing typed double on the way
            if (ob >= 0) {
                const long long* src = (const long long*)(f + (((size_t)r * n_i + ob) * L + q) * 3);
                b1 = src[0], b2 = src[1], b3 = src[2];
            }
            zs[(size_t)j * L + qr] = Cx<R>::make(d2f_bits(b1), d2f_bits(b2));
            wp[j & 1] = d2f_bits(b3);
            continue;
        }
        double f1 = 0.0, f2 = 0.0, f3 = 0.0;
        if (ob >= 0) {
            const double* src = f + (((size_t)r * n_i + ob) * L + q) * 3;
            f1 = src[0], f2 = src[1], f3 = src[2];
        }
        {
            zs[(size_t)j * L + qr] = Cx<R>::make((R)f1, (R)f2);
            wp[j & 1] = (R)f3;
        }
    }
    if (kF32) {
        // one warp per column: lane-strided FP64 sums, then a fixed shuffle tree (deterministic)
        const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
        for (int j = warp; j < NC; j += nw) {
            const int ob = perm[b0 + j];
            double a0 = 0.0, a1 = 0.0, a2 = 0.0;
            if (ob >= 0)
                for (int q = lane; q < L; q += 32) {
                    const double* src = f + (((size_t)r * n_i + ob) * L + q) * 3;
                    a0 += src[0], a1 += src[1], a2 += src[2];
                }
            for (int o = 16; o > 0; o >>= 1) {
                a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            }
            if (lane == 0) s0[j][0] = a0, s0[j][1] = a1, s0[j][2] = a2;
        }
    }
    __syncthreads();
    fft_block<R>(zs, NC + NC / 2, L, logL, tw, false);
    // unpack and store six-vectors for k = 0..L/2
    for (int t = threadIdx.x; t < NC * K; t += blockDim.x) {
        const int k = t >> logNC, j = t & (NC - 1);
        const int km = (L - k) & (L - 1);
        const T2 Z = zs[(size_t)j * L + k], Zm = zs[(size_t)j * L + km];
        const T2 Wv = ws[(size_t)(j >> 1) * L + k], Wm = ws[(size_t)(j >> 1) * L + km];
        // F1 = (Z + conj Zm) / 2, F2 = (Z - conj Zm) / (2i)
        double F1r, F1i, F2r, F2i, F3r, F3i;
        if constexpr (kF32) {
            // unpack in FP32, widen exactly
            F1r = f2d_int(0.5f * (Z.x + Zm.x)), F1i = f2d_int(0.5f * (Z.y - Zm.y));
            F2r = f2d_int(0.5f * (Z.y + Zm.y)), F2i = f2d_int(-0.5f * (Z.x - Zm.x));
            if ((j & 1) == 0) {
                F3r = f2d_int(0.5f * (Wv.x + Wm.x)), F3i = f2d_int(0.5f * (Wv.y - Wm.y));
            } else {
                F3r = f2d_int(0.5f * (Wv.y + Wm.y)), F3i = f2d_int(-0.5f * (Wv.x - Wm.x));
            }
            if (k == 0) F1r = s0[j][0], F2r = s0[j][1], F3r = s0[j][2], F1i = F2i = F3i = 0.0;
        } else {
            F1r = 0.5 * ((double)Z.x + Zm.x), F1i = 0.5 * ((double)Z.y - Zm.y);
            F2r = 0.5 * ((double)Z.y + Zm.y), F2i = -0.5 * ((double)Z.x - Zm.x);
            if ((j & 1) == 0) {
                F3r = 0.5 * ((double)Wv.x + Wm.x), F3i = 0.5 * ((double)Wv.y - Wm.y);
            } else {
                F3r = 0.5 * ((double)Wv.y + Wm.y), F3i = -0.5 * ((double)Wv.x - Wm.x);
            }
        }
        double* o = fh + (((size_t)r * K + k) * NIpad + b0 + j) * 6;
        if (perm[b0 + j] < 0) {
            o[0] = o[1] = o[2] = o[3] = o[4] = o[5] = 0.0;
            continue;
        }
        o[0] = F1r;
        o[1] = F2r;
        o[2] = F3i;
        o[3] = F1i;
        o[4] = F2i;
        o[5] = -F3r;
    }
}

// Neutral projection in the mode domain: mean_c = sum_b F_c(b, 0) / (n_i L);
// F_c(b, 0) -= L mean_c for every real column.  One CTA of 256 threads per
// right-hand side; fixed-order reduction (deterministic).
__device__ __forceinline__ void project_rhs(double* __restrict__ fh, const int* __restrict__ perm, int n_i, int K,
                                            int NIpad, int r) {
    __shared__ double red[3][256];
    double* row = fh + (size_t)r * K * NIpad * 6;  // k = 0
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < NIpad; b += blockDim.x) {
        s0 += row[(size_t)b * 6 + 0];
        s1 += row[(size_t)b * 6 + 1];
        s2 -= row[(size_t)b * 6 + 5];
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int c = 0; c < 3; c++) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    // L * mean = sum / n_i
    const double m0 = red[0][0] / (double)n_i, m1 = red[1][0] / (double)n_i, m2 = red[2][0] / (double)n_i;
    for (int b = threadIdx.x; b < NIpad; b += blockDim.x) {
        if (perm[b] < 0) continue;
        row[(size_t)b * 6 + 0] -= m0;
        row[(size_t)b * 6 + 1] -= m1;
        row[(size_t)b * 6 + 5] += m2;
    }
}

// Inverse transform + epilogue of NC pad columns (block blk of right-hand side
// r); with want_part the block's per-component sums go to part[r][blk].
template <typename R>
__device__ __forceinline__ void inv_block(const double* __restrict__ uh, const int* __restrict__ perm,
                                          const double2* __restrict__ tw, double* __restrict__ u,
                                          double* __restrict__ part, int n_p, int L, int logL, int K, int NPpad,
                                          int NC, double alpha_over_L, double beta, int want_part, int blk, int n_blk,
                                          int r, void* sraw, const double* __restrict__ alpha_dev = nullptr,
                                          double alpha_dev_scale = 0.0, double* __restrict__ gmax_part = nullptr,
                                          const float* __restrict__ uh32 = nullptr) {
    using T2 = typename Cx<R>::T;
    constexpr bool kF32 = sizeof(R) == 4;
    const int logNC = __ffs(NC) - 1;  // NC and L are powers of two: shifts, no integer division
    const int a0 = blk * NC;
    // per-rhs multiplier from device memory (the relaxed update), or the launch's alpha / L
    if (alpha_dev) alpha_over_L = alpha_dev_scale * alpha_dev[r];
    // gmax_part: only the block's largest |alpha/L sum_k ...| is recorded, nothing is written
    const bool max_only = gmax_part != nullptr;
    float mx32 = 0.f;
    double mx64 = 0.0;
    const bool has_beta = beta != 0.0;
    T2* zs = (T2*)sraw;
    T2* ws = zs + (size_t)NC * L;
    __shared__ double u0[kF32 ? 64 : 1][3];  // FP64 k = 0 term per column (FP32 form)
    const int Lh = L >> 1;
    for (int t = threadIdx.x; t < NC * K; t += blockDim.x) {
        const int k = t >> logNC, j = t & (NC - 1);
        const double* src = uh + (((size_t)r * K + k) * NPpad + a0 + j) * 6;
        if constexpr (kF32) {
            // k = 0 kept in FP64 beside the transform; the rest converted on the integer pipes
            float U1r, U1i, U2r, U2i;
            if (k == 0) {
                u0[j][0] = src[0], u0[j][1] = src[1];
                U1r = U2r = U1i = U2i = 0.f;
            } else if (uh32) {  // the tensor-core forms' modes k >= 1, kept in FP32
                const float* s32 = uh32 + (((size_t)r * K + k) * NPpad + a0 + j) * 6;
                U1r = s32[0], U2r = s32[1];
                U1i = k == Lh ? 0.f : s32[3];
                U2i = k == Lh ? 0.f : s32[4];
            } else {
                const long long* sb = (const long long*)src;  // raw FP64 words
                U1r = d2f_bits(sb[0]), U2r = d2f_bits(sb[1]);
                U1i = k == Lh ? 0.f : d2f_bits(sb[3]);
                U2i = k == Lh ? 0.f : d2f_bits(sb[4]);
            }
            zs[(size_t)j * L + bitrev(k, logL)] = Cx<R>::make(U1r - U2i, U1i + U2r);
            if (k != 0 && k != Lh) zs[(size_t)j * L + bitrev(L - k, logL)] = Cx<R>::make(U1r + U2i, U2r - U1i);
            continue;
        }
        const double x0 = src[0], x1 = src[1], y0 = src[3], y1 = src[4];
        // U1 = x0 + i y0, U2 = x1 + i y1 (U3 is handled per column pair below)
        double U1r = x0, U1i = y0, U2r = x1, U2i = y1;
        if (k == 0 || k == Lh) U1i = U2i = 0.0;
        // Z(k) = U1 + i U2 ; Z(L-k) = conj U1 + i conj U2
        zs[(size_t)j * L + bitrev(k, logL)] = Cx<R>::make((R)(U1r - U2i), (R)(U1i + U2r));
        if (k != 0 && k != Lh)
            zs[(size_t)j * L + bitrev(L - k, logL)] = Cx<R>::make((R)(U1r + U2i), (R)(U2r - U1i));
    }
    // W = U3(even column) + i U3(odd column), with U3 = -y2 + i x2: thread per (k, column pair)
    for (int t = threadIdx.x; t < (NC / 2) * K; t += blockDim.x) {
        const int k = t >> (logNC - 1), jp = t & ((NC >> 1) - 1);
        const double* se = uh + (((size_t)r * K + k) * NPpad + a0 + 2 * jp) * 6;
        const double* so = se + 6;
        if constexpr (kF32) {
            float Er, Ei, Or, Oi;
            if (k == 0) {
                u0[2 * jp][2] = -se[5], u0[2 * jp + 1][2] = -so[5];
                Er = Ei = Or = Oi = 0.f;
            } else if (uh32) {
                const float* e32 = uh32 + (((size_t)r * K + k) * NPpad + a0 + 2 * jp) * 6;
                const float* o32 = e32 + 6;
                Er = -e32[5], Or = -o32[5];
                Ei = k == Lh ? 0.f : e32[2];
                Oi = k == Lh ? 0.f : o32[2];
            } else {
                const long long *eb = (const long long*)se, *ob = (const long long*)so;
                Er = -d2f_bits(eb[5]), Or = -d2f_bits(ob[5]);
                Ei = k == Lh ? 0.f : d2f_bits(eb[2]);
                Oi = k == Lh ? 0.f : d2f_bits(ob[2]);
            }
            ws[(size_t)jp * L + bitrev(k, logL)] = Cx<R>::make(Er - Oi, Ei + Or);
            if (k != 0 && k != Lh) ws[(size_t)jp * L + bitrev(L - k, logL)] = Cx<R>::make(Er + Oi, Or - Ei);
            continue;
        }
        double Er = -se[5], Ei = se[2], Or = -so[5], Oi = so[2];
        if (k == 0 || k == Lh) Ei = Oi = 0.0;
        // W(k) = E + i O ; W(L-k) = conj E + i conj O
        ws[(size_t)jp * L + bitrev(k, logL)] = Cx<R>::make((R)(Er - Oi), (R)(Ei + Or));
        if (k != 0 && k != Lh) ws[(size_t)jp * L + bitrev(L - k, logL)] = Cx<R>::make((R)(Er + Oi), (R)(Or - Ei));
    }
    __syncthreads();
    fft_block<R>(zs, NC + NC / 2, L, logL, tw, true);
    double ps0 = 0.0, ps1 = 0.0, ps2 = 0.0;
    if constexpr (kF32) {
        // the k >= 1 modes sum to zero along the line: remove the mean their FP32
        // transform picked up (summed in double-float), so the k = 0 band keeps FP64
        // accuracy; uk[j][c] = (alpha / L) (U_c(0) - mean) in FP64
        __shared__ double uk[64][3];
        const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
        for (int j = warp; j < NC; j += nw) {
            float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
            for (int p = lane; p < L; p += 32) {
                const T2 z = zs[(size_t)j * L + p];
                const T2 w = ws[(size_t)(j >> 1) * L + p];
                df_acc(z.x, h0, l0), df_acc(z.y, h1, l1), df_acc((j & 1) ? w.y : w.x, h2, l2);
            }
            double a0 = f2d_int(h0) + f2d_int(l0), a1 = f2d_int(h1) + f2d_int(l1), a2 = f2d_int(h2) + f2d_int(l2);
            for (int o = 16; o > 0; o >>= 1) {
                a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            }
            if (lane == 0) {
                uk[j][0] = alpha_over_L * (u0[j][0] - a0 / L);
                uk[j][1] = alpha_over_L * (u0[j][1] - a1 / L);
                uk[j][2] = alpha_over_L * (u0[j][2] - a2 / L);
            }
        }
        __syncthreads();
        const float af = (float)alpha_over_L;
        for (int t = threadIdx.x; t < NC * L; t += blockDim.x) {
            const int j = t >> logL, p = t & (L - 1);
            const int oa = perm[a0 + j];
            if (oa < 0) continue;
            const T2 z = zs[(size_t)j * L + p];
            const T2 w = ws[(size_t)(j >> 1) * L + p];
            if (max_only) {
                // the cap needs |g| to FP32 accuracy: sum in FP32, no FP64 work per element
                const float g0 = af * z.x + (float)uk[j][0], g1 = af * z.y + (float)uk[j][1];
                const float g2 = af * ((j & 1) ? w.y : w.x) + (float)uk[j][2];
                mx32 = fmaxf(mx32, fmaxf(fabsf(g0), fmaxf(fabsf(g1), fabsf(g2))));
                continue;
            }
            double* dst = u + (((size_t)r * n_p + oa) * L + p) * 3;
            double o0 = f2d_int(af * z.x) + uk[j][0];
            double o1 = f2d_int(af * z.y) + uk[j][1];
            double o2 = f2d_int(af * ((j & 1) ? w.y : w.x)) + uk[j][2];
            if (has_beta) {
                o0 = fma(beta, dst[0], o0);
                o1 = fma(beta, dst[1], o1);
                o2 = fma(beta, dst[2], o2);
            }
            dst[0] = o0;
            dst[1] = o1;
            dst[2] = o2;
            if (want_part) ps0 += o0, ps1 += o1, ps2 += o2;
        }
    } else {
        for (int t = threadIdx.x; t < NC * L; t += blockDim.x) {
            const int j = t >> logL, p = t & (L - 1);
            const int oa = perm[a0 + j];
            if (oa < 0) continue;
            const T2 z = zs[(size_t)j * L + p];
            const T2 w = ws[(size_t)(j >> 1) * L + p];
            const double z0 = z.x, z1 = z.y, v3 = (j & 1) ? w.y : w.x;
            double o0 = alpha_over_L * z0, o1 = alpha_over_L * z1, o2 = alpha_over_L * v3;
            if (max_only) {
                mx64 = fmax(mx64, fmax(fabs(o0), fmax(fabs(o1), fabs(o2))));
                continue;
            }
            double* dst = u + (((size_t)r * n_p + oa) * L + p) * 3;
            if (has_beta) {
                o0 = fma(beta, dst[0], o0);
                o1 = fma(beta, dst[1], o1);
                o2 = fma(beta, dst[2], o2);
            }
            dst[0] = o0;
            dst[1] = o1;
            dst[2] = o2;
            ps0 += o0, ps1 += o1, ps2 += o2;
        }
    }
    if (max_only) {
        __shared__ double redm[256];
        redm[threadIdx.x] = kF32 ? (double)mx32 : mx64;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) redm[threadIdx.x] = fmax(redm[threadIdx.x], redm[threadIdx.x + w]);
            __syncthreads();
        }
        if (threadIdx.x == 0) gmax_part[(size_t)r * n_blk + blk] = redm[0];
        return;
    }
    if (want_part) {
        __shared__ double red[3][256];
        red[0][threadIdx.x] = ps0;
        red[1][threadIdx.x] = ps1;
        red[2][threadIdx.x] = ps2;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w)
                for (int c = 0; c < 3; c++) red[c][threadIdx.x] += red[c][threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double* pp = part + ((size_t)r * n_blk + blk) * 3;
            pp[0] = red[0][0], pp[1] = red[1][0], pp[2] = red[2][0];
        }
    }
}

// ---- FP32 line transforms in the Stockham form ---------------------------------
// The FP32 forms' transforms when L <= 2048 and the caller's arrays are 16-byte
// aligned: natural order in and out, radix-8 passes in shared memory (4 passes
// at L = 1024 instead of 10 radix-2 stages; padded index, no bank conflicts),
// each lane of a warp moving two rows of a column [L][3] as three 16-byte
// words, the FP64 k = 0 sums taken from the same loads, 16-byte stores of the
// six-vectors.  The arithmetic per element is that of the radix-2 form: FP32
// transform, k = 0 in FP64.  twl[m] = exp(-2 pi i m / L), m < L, in FP32.
__device__ __forceinline__ void fwd_block_s(const double* __restrict__ f, const int* __restrict__ perm,
                                            const float2* __restrict__ twl, const Fft1D& F, double* __restrict__ fh,
                                            int n_i, int L, int K, int NIpad, int NC, int blk, int r, void* sraw) {
    const int nseq = NC + NC / 2, logNC = __ffs(NC) - 1, Lh = L >> 1;
    float2* A = (float2*)sraw;
    float2* B = A + fft::padded(nseq * L);
    __shared__ double s0[64][3];  // FP64 column sums = the k = 0 mode
    const int b0 = blk * NC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // wpc warps share a column (all warps busy when the CTA holds fewer columns than warps)
    const int wpc = nw > NC ? nw / NC : 1, sub = warp % wpc;
    __shared__ double s0p[8][3];  // per-warp partial sums when a column is shared
    for (int j = warp / wpc; j < NC; j += nw / wpc) {
        const int ob = perm[b0 + j];
        const double2* src = ob >= 0 ? (const double2*)(f + ((size_t)r * n_i + ob) * L * 3) : nullptr;
        const int zb = j * L, wb = (NC + (j >> 1)) * L, half = j & 1;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int m = lane + 32 * sub; m < Lh; m += 32 * wpc) {
            double2 v0 = make_double2(0.0, 0.0), v1 = v0, v2 = v0;
            if (src) v0 = src[3 * m], v1 = src[3 * m + 1], v2 = src[3 * m + 2];
            // row 2m: (v0.x, v0.y, v1.x); row 2m + 1: (v1.y, v2.x, v2.y)
            a0 += v0.x, a0 += v1.y, a1 += v0.y, a1 += v2.x, a2 += v1.x, a2 += v2.y;
            A[fft::sx(zb + 2 * m)] = make_float2(d2f_int(v0.x), d2f_int(v0.y));
            A[fft::sx(zb + 2 * m + 1)] = make_float2(d2f_int(v1.y), d2f_int(v2.x));
            ((float*)&A[fft::sx(wb + 2 * m)])[half] = d2f_int(v1.x);
            ((float*)&A[fft::sx(wb + 2 * m + 1)])[half] = d2f_int(v2.y);
        }
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
            if (wpc == 1) s0[j][0] = a0, s0[j][1] = a1, s0[j][2] = a2;
            else s0p[warp][0] = a0, s0p[warp][1] = a1, s0p[warp][2] = a2;
        }
    }
    __syncthreads();
    if (wpc > 1 && threadIdx.x < NC * 3) {  // the warps of a column in a fixed order (deterministic)
        const int j = threadIdx.x / 3, c = threadIdx.x % 3;
        double a = 0.0;
        for (int w = 0; w < wpc; w++) a += s0p[j * wpc + w][c];
        s0[j][c] = a;
    }
    const float2* Y = fft::fft_smem<false>(A, B, nseq, F, twl);
    for (int t = threadIdx.x; t < NC * K; t += blockDim.x) {
        const int k = t >> logNC, j = t & (NC - 1);
        double2* o = (double2*)(fh + (((size_t)r * K + k) * NIpad + b0 + j) * 6);
        if (perm[b0 + j] < 0) {
            o[0] = o[1] = o[2] = make_double2(0.0, 0.0);
            continue;
        }
        const int km = (L - k) & (L - 1), wb = (NC + (j >> 1)) * L;
        const float2 Z = Y[fft::sx(j * L + k)], Zm = Y[fft::sx(j * L + km)];
        const float2 Wv = Y[fft::sx(wb + k)], Wm = Y[fft::sx(wb + km)];
        // F1 = (Z + conj Zm) / 2, F2 = (Z - conj Zm) / (2i); F3 from W the same way (x part or y part)
        double F1r = f2d_int(0.5f * (Z.x + Zm.x)), F1i = f2d_int(0.5f * (Z.y - Zm.y));
        double F2r = f2d_int(0.5f * (Z.y + Zm.y)), F2i = f2d_int(-0.5f * (Z.x - Zm.x));
        double F3r, F3i;
        if ((j & 1) == 0) {
            F3r = f2d_int(0.5f * (Wv.x + Wm.x)), F3i = f2d_int(0.5f * (Wv.y - Wm.y));
        } else {
            F3r = f2d_int(0.5f * (Wv.y + Wm.y)), F3i = f2d_int(-0.5f * (Wv.x - Wm.x));
        }
        if (k == 0) F1r = s0[j][0], F2r = s0[j][1], F3r = s0[j][2], F1i = F2i = F3i = 0.0;
        o[0] = make_double2(F1r, F2r);
        o[1] = make_double2(F3i, F1i);
        o[2] = make_double2(F2i, -F3r);
    }
}

__device__ __forceinline__ void inv_block_s(const double* __restrict__ uh, const int* __restrict__ perm,
                                            const float2* __restrict__ twl, const Fft1D& F, double* __restrict__ u,
                                            double* __restrict__ part, int n_p, int L, int K, int NPpad, int NC,
                                            double alpha_over_L, double beta, int want_part, int blk, int n_blk,
                                            int r, void* sraw, const double* __restrict__ alpha_dev = nullptr,
                                            double alpha_dev_scale = 0.0, double* __restrict__ gmax_part = nullptr,
                                            const float* __restrict__ uh32 = nullptr) {
    const int nseq = NC + NC / 2, logNC = __ffs(NC) - 1, Lh = L >> 1;
    float2* A = (float2*)sraw;
    float2* B = A + fft::padded(nseq * L);
    // FP64 k = 0 term per column, and the column's final k = 0 value: after the two FFT buffers in
    // the dynamic shared memory (sized for this launch's NC, not the largest), so that at L = 1024
    // four CTAs fit on an SM
    double (*u0)[3] = reinterpret_cast<double (*)[3]>(B + fft::padded(nseq * L));
    double (*uk)[3] = u0 + NC;
    const int a0 = blk * NC;
    if (alpha_dev) alpha_over_L = alpha_dev_scale * alpha_dev[r];
    const bool max_only = gmax_part != nullptr;
    const bool has_beta = beta != 0.0;
    // Z = U1 + i U2 per column: Z(k) and Z(L - k) = conj U1 + i conj U2
    for (int t = threadIdx.x; t < NC * K; t += blockDim.x) {
        const int k = t >> logNC, j = t & (NC - 1);
        const double2* src = (const double2*)(uh + (((size_t)r * K + k) * NPpad + a0 + j) * 6);
        if (k == 0) {
            const double2 p0 = src[0];
            u0[j][0] = p0.x, u0[j][1] = p0.y;
            A[fft::sx(j * L)] = make_float2(0.f, 0.f);
            continue;
        }
        float U1r, U2r, U1i, U2i;
        if (uh32) {  // the tensor-core forms' modes k >= 1, kept in FP32: (Re V1, Re V2) (Im V3, Im V1) (Im V2, -Re V3)
            const float2* s32 = (const float2*)(uh32 + (((size_t)r * K + k) * NPpad + a0 + j) * 6);
            const float2 q0 = s32[0], q1 = s32[1], q2 = s32[2];
            U1r = q0.x, U2r = q0.y, U1i = k == Lh ? 0.f : q1.y, U2i = k == Lh ? 0.f : q2.x;
        } else {
            const double2 p0 = src[0], p1 = src[1], p2 = src[2];  // (Re V1, Re V2) (Im V3, Im V1) (Im V2, -Re V3)
            U1r = d2f_int(p0.x), U2r = d2f_int(p0.y);
            U1i = k == Lh ? 0.f : d2f_int(p1.y), U2i = k == Lh ? 0.f : d2f_int(p2.x);
        }
        A[fft::sx(j * L + k)] = make_float2(U1r - U2i, U1i + U2r);
        if (k != Lh) A[fft::sx(j * L + L - k)] = make_float2(U1r + U2i, U2r - U1i);
    }
    // W = U3(even column) + i U3(odd column), with U3 = -y2 + i x2
    for (int t = threadIdx.x; t < (NC / 2) * K; t += blockDim.x) {
        const int k = t >> (logNC - 1), jp = t & ((NC >> 1) - 1);
        const double* se = uh + (((size_t)r * K + k) * NPpad + a0 + 2 * jp) * 6;
        const double* so = se + 6;
        const int wb = (NC + jp) * L;
        if (k == 0) {
            u0[2 * jp][2] = -se[5], u0[2 * jp + 1][2] = -so[5];
            A[fft::sx(wb)] = make_float2(0.f, 0.f);
            continue;
        }
        float Er, Or, Ei, Oi;
        if (uh32) {
            const float* e32 = uh32 + (((size_t)r * K + k) * NPpad + a0 + 2 * jp) * 6;
            Er = -e32[5], Or = -e32[11], Ei = k == Lh ? 0.f : e32[2], Oi = k == Lh ? 0.f : e32[8];
        } else {
            Er = -d2f_int(se[5]), Or = -d2f_int(so[5]);
            Ei = k == Lh ? 0.f : d2f_int(se[2]), Oi = k == Lh ? 0.f : d2f_int(so[2]);
        }
        A[fft::sx(wb + k)] = make_float2(Er - Oi, Ei + Or);
        if (k != Lh) A[fft::sx(wb + L - k)] = make_float2(Er + Oi, Or - Ei);
    }
    __syncthreads();
    const float2* Y = fft::fft_smem<true>(A, B, nseq, F, twl);
    // the k >= 1 modes sum to zero along the line: remove the mean their FP32 transform picked up (summed in
    // double-float), so the k = 0 band keeps FP64 accuracy; uk[j][c] = (alpha / L) (U_c(0) - mean) in FP64
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int wpc = nw > NC ? nw / NC : 1, sub = warp % wpc;  // warps per column
    // per-warp partial sums when warps share a column (wpc > 1: each warp then has exactly one column):
    // 3 doubles per warp in the transform's other buffer, free once Y holds the result (at least
    // 1.5 NC L = 192 FP32 complex numbers, 1536 bytes, for L = 2)
    double* scr = (double*)(Y == A ? B : A);
    for (int j = warp / wpc; j < NC; j += nw / wpc) {
        const int wb = (NC + (j >> 1)) * L;
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
        for (int p = lane + 32 * sub; p < L; p += 32 * wpc) {
            const float2 z = Y[fft::sx(j * L + p)];
            const float2 w = Y[fft::sx(wb + p)];
            df_acc(z.x, h0, l0), df_acc(z.y, h1, l1), df_acc((j & 1) ? w.y : w.x, h2, l2);
        }
        double a0_ = f2d_int(h0) + f2d_int(l0), a1_ = f2d_int(h1) + f2d_int(l1), a2_ = f2d_int(h2) + f2d_int(l2);
        for (int o = 16; o > 0; o >>= 1) {
            a0_ += __shfl_xor_sync(0xffffffffu, a0_, o);
            a1_ += __shfl_xor_sync(0xffffffffu, a1_, o);
            a2_ += __shfl_xor_sync(0xffffffffu, a2_, o);
        }
        if (lane == 0) {
            if (wpc == 1) {
                uk[j][0] = alpha_over_L * (u0[j][0] - a0_ / L);
                uk[j][1] = alpha_over_L * (u0[j][1] - a1_ / L);
                uk[j][2] = alpha_over_L * (u0[j][2] - a2_ / L);
            } else {
                scr[3 * warp] = a0_, scr[3 * warp + 1] = a1_, scr[3 * warp + 2] = a2_;
            }
        }
    }
    __syncthreads();
    if (wpc > 1 && threadIdx.x < NC * 3) {  // the warps of a column in a fixed order (deterministic)
        const int j = threadIdx.x / 3, c = threadIdx.x % 3;
        double a = 0.0;
        for (int w = 0; w < wpc; w++) a += scr[3 * (j * wpc + w) + c];
        uk[j][c] = alpha_over_L * (u0[j][c] - a / L);
    }
    __syncthreads();
    const float af = (float)alpha_over_L;
    float mx32 = 0.f;
    double ps0 = 0.0, ps1 = 0.0, ps2 = 0.0;
    for (int j = warp / wpc; j < NC; j += nw / wpc) {
        const int oa = perm[a0 + j];
        if (oa < 0) continue;
        const int zb = j * L, wb = (NC + (j >> 1)) * L, half = j & 1;
        const double k0 = uk[j][0], k1 = uk[j][1], k2 = uk[j][2];
        double2* dst = (double2*)(u + ((size_t)r * n_p + oa) * L * 3);
        for (int m = lane + 32 * sub; m < Lh; m += 32 * wpc) {
            const float2 z0 = Y[fft::sx(zb + 2 * m)], z1 = Y[fft::sx(zb + 2 * m + 1)];
            const float2 w0 = Y[fft::sx(wb + 2 * m)], w1 = Y[fft::sx(wb + 2 * m + 1)];
            const float w0h = half ? w0.y : w0.x, w1h = half ? w1.y : w1.x;
            if (max_only) {
                // the cap needs |g| to FP32 accuracy: sum in FP32, no FP64 work per element
                const float g[6] = {af * z0.x + (float)k0, af * z0.y + (float)k1, af * w0h + (float)k2,
                                    af * z1.x + (float)k0, af * z1.y + (float)k1, af * w1h + (float)k2};
#pragma unroll
                for (int c = 0; c < 6; c++) mx32 = fmaxf(mx32, fabsf(g[c]));
                continue;
            }
            double o[6] = {f2d_int(af * z0.x) + k0, f2d_int(af * z0.y) + k1, f2d_int(af * w0h) + k2,
                           f2d_int(af * z1.x) + k0, f2d_int(af * z1.y) + k1, f2d_int(af * w1h) + k2};
            if (has_beta) {
                const double2 d0 = dst[3 * m], d1 = dst[3 * m + 1], d2 = dst[3 * m + 2];
                o[0] = fma(beta, d0.x, o[0]), o[1] = fma(beta, d0.y, o[1]), o[2] = fma(beta, d1.x, o[2]);
                o[3] = fma(beta, d1.y, o[3]), o[4] = fma(beta, d2.x, o[4]), o[5] = fma(beta, d2.y, o[5]);
            }
            dst[3 * m] = make_double2(o[0], o[1]);
            dst[3 * m + 1] = make_double2(o[2], o[3]);
            dst[3 * m + 2] = make_double2(o[4], o[5]);
            if (want_part) ps0 += o[0], ps0 += o[3], ps1 += o[1], ps1 += o[4], ps2 += o[2], ps2 += o[5];
        }
    }
    // block reductions (the maximum, or the three partial sums): a fixed shuffle tree per warp, then
    // the warps in order; 192 bytes of static shared memory, so shared memory allows a fourth CTA
    __shared__ double red[8][3];
    if (max_only) {
        float m = mx32;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) red[warp][0] = (double)m;
        __syncthreads();
        if (threadIdx.x == 0) {
            double mm = red[0][0];
            for (int w = 1; w < nw; w++) mm = fmax(mm, red[w][0]);
            gmax_part[(size_t)r * n_blk + blk] = mm;
        }
        return;
    }
    if (want_part) {
        for (int o = 16; o > 0; o >>= 1) {
            ps0 += __shfl_xor_sync(0xffffffffu, ps0, o);
            ps1 += __shfl_xor_sync(0xffffffffu, ps1, o);
            ps2 += __shfl_xor_sync(0xffffffffu, ps2, o);
        }
        if (lane == 0) red[warp][0] = ps0, red[warp][1] = ps1, red[warp][2] = ps2;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            for (int w = 0; w < nw; w++) s0 += red[w][0], s1 += red[w][1], s2 += red[w][2];
            double* pp = part + ((size_t)r * n_blk + blk) * 3;
            pp[0] = s0, pp[1] = s1, pp[2] = s2;
        }
    }
}

// Zero mean of the pad displacements (Eq. 23): every CTA reduces the per-CTA
// partial sums in the same fixed order, then subtracts from chunk c of n_chunk.
__device__ __forceinline__ void zero_mean_chunk(double* __restrict__ u, const double* __restrict__ part, int n_part,
                                                int n_p, int L, int r, int c, int n_chunk) {
    __shared__ double mean[3];
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        const double* pp = part + (size_t)r * n_part * 3;
        for (int t = 0; t < n_part; t++) s0 += pp[3 * t], s1 += pp[3 * t + 1], s2 += pp[3 * t + 2];
        const double inv = 1.0 / ((double)n_p * (double)L);
        mean[0] = s0 * inv, mean[1] = s1 * inv, mean[2] = s2 * inv;
    }
    __syncthreads();
    const size_t n = (size_t)n_p * L * 3;
    double* ur = u + (size_t)r * n;
    for (size_t i = (size_t)c * blockDim.x + threadIdx.x; i < n; i += (size_t)n_chunk * blockDim.x)
        ur[i] -= mean[i % 3];
}

// ---- one launch per plan ------------------------------------------------------
template <typename R>
__global__ void k_forward(const double* __restrict__ f, const int* __restrict__ perm, const double2* __restrict__ tw,
                          double* __restrict__ fh, int n_i, int L, int logL, int K, int NIpad, int NC) {
    extern __shared__ double2 sbuf[];
    fwd_block<R>(f, perm, tw, fh, n_i, L, logL, K, NIpad, NC, blockIdx.x, blockIdx.y, sbuf);
}
__global__ void k_project(double* __restrict__ fh, const int* __restrict__ perm, int n_i, int K, int NIpad) {
    project_rhs(fh, perm, n_i, K, NIpad, blockIdx.y);
}
template <typename R>
__global__ void k_inverse(const double* __restrict__ uh, const int* __restrict__ perm, const double2* __restrict__ tw,
                          double* __restrict__ u, double* __restrict__ part, int n_p, int L, int logL, int K, int NPpad,
                          int NC, double alpha_over_L, double beta, int want_part, const double* __restrict__ alpha_dev,
                          double alpha_dev_scale, double* __restrict__ gmax_part, const float* __restrict__ uh32) {
    extern __shared__ double2 sbuf[];
    inv_block<R>(uh, perm, tw, u, part, n_p, L, logL, K, NPpad, NC, alpha_over_L, beta, want_part, blockIdx.x,
                 gridDim.x, blockIdx.y, sbuf, alpha_dev, alpha_dev_scale, gmax_part, uh32);
}
__global__ void k_forward_s(const double* __restrict__ f, const int* __restrict__ perm, const float2* __restrict__ twl,
                            Fft1D F, double* __restrict__ fh, int n_i, int L, int K, int NIpad, int NC) {
    extern __shared__ double2 sbuf[];
    fwd_block_s(f, perm, twl, F, fh, n_i, L, K, NIpad, NC, blockIdx.x, blockIdx.y, sbuf);
}
__global__ void k_inverse_s(const double* __restrict__ uh, const int* __restrict__ perm, const float2* __restrict__ twl,
                            Fft1D F, double* __restrict__ u, double* __restrict__ part, int n_p, int L, int K, int NPpad,
                            int NC, double alpha_over_L, double beta, int want_part, const double* __restrict__ alpha_dev,
                            double alpha_dev_scale, double* __restrict__ gmax_part, const float* __restrict__ uh32) {
    extern __shared__ double2 sbuf[];
    inv_block_s(uh, perm, twl, F, u, part, n_p, L, K, NPpad, NC, alpha_over_L, beta, want_part, blockIdx.x, gridDim.x,
                blockIdx.y, sbuf, alpha_dev, alpha_dev_scale, gmax_part, uh32);
}
__global__ void k_zero_mean(double* __restrict__ u, const double* __restrict__ part, int n_part, int n_p, int L) {
    zero_mean_chunk(u, part, n_part, n_p, L, blockIdx.y, blockIdx.x, gridDim.x);
}

// ---- batched over plans: items (instance, block, right-hand side) ---------------
template <typename R>
__global__ void k_batch_forward(const LineArgs* __restrict__ la, const int4* __restrict__ items) {
    extern __shared__ double2 sbuf[];
    const int4 w = items[blockIdx.x];
    const LineArgs A = la[w.x];
    if (sizeof(R) == 4 && A.stockham)
        fwd_block_s(A.f, A.perm_i, A.twl, A.F, A.fh, A.n_i, A.L, A.K, A.NIpad, A.NC, w.y, w.z, sbuf);
    else
        fwd_block<R>(A.f, A.perm_i, A.tw, A.fh, A.n_i, A.L, A.logL, A.K, A.NIpad, A.NC, w.y, w.z, sbuf);
}
__global__ void k_batch_project(const LineArgs* __restrict__ la, const int4* __restrict__ items) {
    const int4 w = items[blockIdx.x];
    const LineArgs A = la[w.x];
    project_rhs(A.fh, A.perm_i, A.n_i, A.K, A.NIpad, w.z);
}
template <typename R>
__global__ void k_batch_inverse(const LineArgs* __restrict__ la, const int4* __restrict__ items, double alpha,
                                double beta, int want_part) {
    extern __shared__ double2 sbuf[];
    const int4 w = items[blockIdx.x];
    const LineArgs A = la[w.x];
    if (sizeof(R) == 4 && A.stockham)
        inv_block_s(A.uh, A.perm_p, A.twl, A.F, A.u, A.part, A.n_p, A.L, A.K, A.NPpad, A.NC, alpha / (double)A.L,
                    beta, want_part, w.y, A.NPpad / A.NC, w.z, sbuf, nullptr, 0.0, nullptr, A.uh32);
    else
        inv_block<R>(A.uh, A.perm_p, A.tw, A.u, A.part, A.n_p, A.L, A.logL, A.K, A.NPpad, A.NC, alpha / (double)A.L,
                     beta, want_part, w.y, A.NPpad / A.NC, w.z, sbuf, nullptr, 0.0, nullptr, A.uh32);
}
__global__ void k_batch_zero_mean(const LineArgs* __restrict__ la, const int4* __restrict__ items) {
    const int4 w = items[blockIdx.x];  // (instance, chunk, r, n_chunk)
    const LineArgs A = la[w.x];
    zero_mean_chunk(A.u, A.part, A.NPpad / A.NC, A.n_p, A.L, w.z, w.y, w.w);
}

size_t line_smem(int L, int NC) { return (size_t)(NC + NC / 2) * L * sizeof(double2); }
// the Stockham FP32 form: two padded buffers of FP32 complex numbers
size_t line_smem_s(int L, int NC) {
    return (size_t)2 * fft::padded((NC + NC / 2) * L) * sizeof(float2) + (size_t)2 * NC * 3 * sizeof(double);
}

}  // namespace

bool line_stockham(int L, const void* a, const void* b) {
    return L >= 2 && L <= kLineStockhamMaxL && ((uintptr_t)a & 15) == 0 && ((uintptr_t)b & 15) == 0;
}

cudaError_t launch_forward(Plan& P, const double* f, int n_rhs, bool project, cudaStream_t st) {
    const int NC = line_cols(P.L);
    const size_t smem = line_smem(P.L, NC);
    cudaError_t e;
    // opt in above the default dynamic limit (the kernel's static arrays count towards 48 KB)
    dim3 grid(P.NIpad / NC, n_rhs);
    if (line_fp32(P.precision) && line_stockham(P.L, f, P.d_fh)) {
        const size_t ss = line_smem_s(P.L, NC);
        if ((e = cudaFuncSetAttribute(k_forward_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss))) return e;
        k_forward_s<<<grid, 256, ss, st>>>(f, P.d_perm_i, P.d_twl, P.line_fft, P.d_fh, P.n_i, P.L, P.K, P.NIpad, NC);
    } else if (line_fp32(P.precision)) {
        if ((e = cudaFuncSetAttribute(k_forward<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k_forward<float><<<grid, 256, smem / 2, st>>>(f, P.d_perm_i, P.d_tw, P.d_fh, P.n_i, P.L, P.logL, P.K, P.NIpad, NC);
    } else {
        if ((e = cudaFuncSetAttribute(k_forward<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k_forward<double><<<grid, 256, smem, st>>>(f, P.d_perm_i, P.d_tw, P.d_fh, P.n_i, P.L, P.logL, P.K, P.NIpad, NC);
    }
    if ((e = cudaGetLastError())) return e;
    if (project) {
        k_project<<<dim3(1, n_rhs), 256, 0, st>>>(P.d_fh, P.d_perm_i, P.n_i, P.K, P.NIpad);
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_inverse(Plan& P, double* u, int n_rhs, double alpha, double beta, bool zero_mean,
                           cudaStream_t st, const double* alpha_dev, double alpha_dev_scale, double* gmax_part) {
    const int NC = line_cols(P.L);
    const size_t smem = line_smem(P.L, NC);
    cudaError_t e;
    const int nb = P.NPpad / NC;
    dim3 grid(nb, n_rhs);
    // the tensor-core forms leave their modes k >= 1 in FP32 (k = 0 in the FP64 buffer)
    const float* uh32 = is_tensor_precision(P.precision) ? P.d_uh32 : nullptr;
    if (line_fp32(P.precision) && line_stockham(P.L, u, P.d_uh)) {
        const size_t ss = line_smem_s(P.L, NC);
        if ((e = cudaFuncSetAttribute(k_inverse_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss))) return e;
        k_inverse_s<<<grid, 256, ss, st>>>(P.d_uh, P.d_perm_p, P.d_twl, P.line_fft, u, P.d_part, P.n_p, P.L, P.K, P.NPpad,
                                           NC, alpha / (double)P.L, beta, zero_mean ? 1 : 0, alpha_dev, alpha_dev_scale,
                                           gmax_part, uh32);
    } else if (line_fp32(P.precision)) {
        if ((e = cudaFuncSetAttribute(k_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k_inverse<float><<<grid, 256, smem / 2, st>>>(P.d_uh, P.d_perm_p, P.d_tw, u, P.d_part, P.n_p, P.L, P.logL, P.K,
                                                      P.NPpad, NC, alpha / (double)P.L, beta, zero_mean ? 1 : 0,
                                                      alpha_dev, alpha_dev_scale, gmax_part, uh32);
    } else {
        if ((e = cudaFuncSetAttribute(k_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k_inverse<double><<<grid, 256, smem, st>>>(P.d_uh, P.d_perm_p, P.d_tw, u, P.d_part, P.n_p, P.L, P.logL, P.K,
                                                   P.NPpad, NC, alpha / (double)P.L, beta, zero_mean ? 1 : 0,
                                                   alpha_dev, alpha_dev_scale, gmax_part, nullptr);
    }
    if ((e = cudaGetLastError())) return e;
    if (zero_mean && !gmax_part) {
        const size_t n = (size_t)P.n_p * P.L * 3;
        int blocks = (int)std::min<size_t>((n + 255) / 256, 4 * 152);
        k_zero_mean<<<dim3(blocks, n_rhs), 256, 0, st>>>(u, P.d_part, nb, P.n_p, P.L);
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

LineArgs make_line_args(const Plan& P, const double* f, double* u) {
    LineArgs A;
    A.f = f, A.u = u, A.fh = P.d_fh, A.uh = P.d_uh, A.perm_i = P.d_perm_i, A.perm_p = P.d_perm_p, A.tw = P.d_tw;
    A.part = P.d_part;
    A.n_i = P.n_i, A.n_p = P.n_p, A.L = P.L, A.logL = P.logL, A.K = P.K, A.NIpad = P.NIpad, A.NPpad = P.NPpad;
    A.NC = line_cols(P.L);
    A.F = P.line_fft;
    A.twl = P.d_twl;
    A.uh32 = is_tensor_precision(P.precision) ? P.d_uh32 : nullptr;
    A.stockham = line_fp32(P.precision) && line_stockham(P.L, f, P.d_fh) && line_stockham(P.L, u, P.d_uh) ? 1 : 0;
    return A;
}

// Dynamic shared memory one instance's line transforms need in its form (the batch launches with the largest).
size_t line_args_smem(const LineArgs& A, bool fp32) {
    if (!fp32) return line_smem(A.L, A.NC);
    return A.stockham ? line_smem_s(A.L, A.NC) : line_smem(A.L, A.NC) / 2;
}

cudaError_t launch_batch_line(int stage, const LineArgs* d_args, const int4* d_items, int n_items, size_t smem,
                              double alpha, double beta, int want_part, cudaStream_t st, bool fp32) {
    if (n_items == 0) return cudaSuccess;
    cudaError_t e;
    switch (stage) {
        case 0:
            if (fp32) {
                if ((e = cudaFuncSetAttribute(k_batch_forward<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem)))
                    return e;
                k_batch_forward<float><<<n_items, 256, smem, st>>>(d_args, d_items);
            } else {
                if ((e = cudaFuncSetAttribute(k_batch_forward<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem)))
                    return e;
                k_batch_forward<double><<<n_items, 256, smem, st>>>(d_args, d_items);
            }
            break;
        case 1:
            k_batch_project<<<n_items, 256, 0, st>>>(d_args, d_items);
            break;
        case 2:
            if (fp32) {
                if ((e = cudaFuncSetAttribute(k_batch_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem)))
                    return e;
                k_batch_inverse<float><<<n_items, 256, smem, st>>>(d_args, d_items, alpha, beta, want_part);
            } else {
                if ((e = cudaFuncSetAttribute(k_batch_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem)))
                    return e;
                k_batch_inverse<double><<<n_items, 256, smem, st>>>(d_args, d_items, alpha, beta, want_part);
            }
            break;
        default:
            k_batch_zero_mean<<<n_items, 256, 0, st>>>(d_args, d_items);
            break;
    }
    return cudaGetLastError();
}

}  // namespace fbc
