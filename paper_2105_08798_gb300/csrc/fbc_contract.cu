// Per-mode contraction (the hot loop):
//     U(a, k) = sum_b g^k(x_a - x_b) F(b, k)
// for every pad column a, wavenumber k and right-hand side (Sec. 3.2,
// Eqs. 37-38, diagonalised along the line).  In the six-vector form each
// pair-mode is one real 3x3 matrix M (built from the six table reals) applied
// to two real 3-vectors x and y' (18 fused multiply-adds).
//
// Blocking: a CTA owns one tile of TA spatially compact pad columns at one
// wavenumber and one right-hand side, one thread per pad column.  It walks
// the TB-column interface tiles; for each, the table entries of every
// difference the tile pair can produce form a small rectangle of the
// difference box (at most W x H entries), which the CTA stages in shared
// memory together with the tile's transformed forces.  Each thread then
// gathers its entries at  idx = base_a - off_b  with base_a fixed per tile
// pair and off_b = x_b + W y_b fixed per interface column.
//
// Precisions: FP64 (DFMA); FP32 (FFMA; the logarithmic k = 0 mode stays on
// the FP64 kernel); F32X2 (double-float: every product and sum carried as an
// unevaluated pair of FP32 numbers -- Dekker's exact product via FMA, Knuth's
// two-sum -- and each interface tile's partial folded into a double-float
// running total, FP64-accurate on the FP32 pipes).
#include <cuda.h>  // CUtensorMap and its encoder's types (the encoder is reached through the runtime)

#include "fbc_internal.cuh"
#include "fbc_tc.cuh"

namespace fbc {
namespace {


template <int TA, int TB>
__device__ __forceinline__ void tile_fp64(const ContractArgs& A, int tA, int k, int r, void* smem_raw) {
    double* smem64 = (double*)smem_raw;
    const int HW = A.H * A.W;
    double* s_tab = smem64;              // [6][HW]
    double* s_f = s_tab + 6 * HW;        // [TB][6]
    int* s_off = (int*)(s_f + TB * 6);   // [TB]
    const int a = tA * TA + threadIdx.x;
    const int2 xa = A.xy_p[a];
    const int4 bA = A.bbox_a[tA];
    double acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0, acc4 = 0, acc5 = 0;
    const double* fk = A.fh + ((size_t)r * A.K + k) * A.NIpad * 6;
    const double* tk = A.tab + (size_t)(k - A.kbase) * A.Dy * A.Dx * 6;
    for (int tB = 0; tB < A.n_tb; tB++) {
        const int4 bB = A.bbox_b[tB];
        const int ox = bA.x - bB.y, oy = bA.z - bB.w;
        __syncthreads();
        for (int e = threadIdx.x; e < HW; e += TA) {
            const int iy = e / A.W, ix = e - iy * A.W;
            const int gx = ox + ix - A.box_x0, gy = oy + iy - A.box_y0;
            double2 v0 = make_double2(0, 0), v1 = v0, v2 = v0;
            if (gx < A.Dx && gy < A.Dy) {
                const double2* src = (const double2*)(tk + ((size_t)gy * A.Dx + gx) * 6);
                v0 = __ldg(src), v1 = __ldg(src + 1), v2 = __ldg(src + 2);
            }
            s_tab[0 * HW + e] = v0.x, s_tab[1 * HW + e] = v0.y;
            s_tab[2 * HW + e] = v1.x, s_tab[3 * HW + e] = v1.y;
            s_tab[4 * HW + e] = v2.x, s_tab[5 * HW + e] = v2.y;
        }
        for (int e = threadIdx.x; e < TB * 6; e += TA) s_f[e] = fk[(size_t)tB * TB * 6 + e];
        for (int e = threadIdx.x; e < TB; e += TA) s_off[e] = A.off_i[tB * TB + e];
        __syncthreads();
        const int base = (xa.x - ox) + A.W * (xa.y - oy);
#pragma unroll 4
        for (int j = 0; j < TB; j++) {
            const int idx = base - s_off[j];
            const double a11 = s_tab[idx], a12 = s_tab[HW + idx], a22 = s_tab[2 * HW + idx];
            const double a33 = s_tab[3 * HW + idx], b13 = s_tab[4 * HW + idx], b23 = s_tab[5 * HW + idx];
            const double* fj = s_f + j * 6;
            const double x0 = fj[0], x1 = fj[1], x2 = fj[2], y0 = fj[3], y1 = fj[4], y2 = fj[5];
            acc0 = fma(a11, x0, fma(a12, x1, fma(-b13, x2, acc0)));
            acc1 = fma(a12, x0, fma(a22, x1, fma(-b23, x2, acc1)));
            acc2 = fma(b13, x0, fma(b23, x1, fma(a33, x2, acc2)));
            acc3 = fma(a11, y0, fma(a12, y1, fma(-b13, y2, acc3)));
            acc4 = fma(a12, y0, fma(a22, y1, fma(-b23, y2, acc4)));
            acc5 = fma(b13, y0, fma(b23, y1, fma(a33, y2, acc5)));
        }
    }
    double* o = A.uh + (((size_t)r * A.K + k) * A.NPpad + a) * 6;
    o[0] = acc0, o[1] = acc1, o[2] = acc2, o[3] = acc3, o[4] = acc4, o[5] = acc5;
}

template <int TA, int TB>
__device__ __forceinline__ void tile_fp32(const ContractArgs& A, int tA, int k, int r, void* smem_raw) {
    float* smem32 = (float*)smem_raw;
    const int HW = A.H * A.W;
    float* s_tab = smem32;              // [6][HW]
    float* s_f = s_tab + 6 * HW;        // [TB][6]
    int* s_off = (int*)(s_f + TB * 6);  // [TB]
    const int a = tA * TA + threadIdx.x;
    const int2 xa = A.xy_p[a];
    const int4 bA = A.bbox_a[tA];
    float acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0, acc4 = 0, acc5 = 0;
    const double* fk = A.fh + ((size_t)r * A.K + k) * A.NIpad * 6;
    const float* tk = A.tab32 + (size_t)(k - A.kbase) * A.Dy * A.Dx * 6;
    for (int tB = 0; tB < A.n_tb; tB++) {
        const int4 bB = A.bbox_b[tB];
        const int ox = bA.x - bB.y, oy = bA.z - bB.w;
        __syncthreads();
        for (int e = threadIdx.x; e < HW; e += TA) {
            const int iy = e / A.W, ix = e - iy * A.W;
            const int gx = ox + ix - A.box_x0, gy = oy + iy - A.box_y0;
            float2 v0 = make_float2(0, 0), v1 = v0, v2 = v0;
            if (gx < A.Dx && gy < A.Dy) {
                const float2* src = (const float2*)(tk + ((size_t)gy * A.Dx + gx) * 6);
                v0 = __ldg(src), v1 = __ldg(src + 1), v2 = __ldg(src + 2);
            }
            s_tab[0 * HW + e] = v0.x, s_tab[1 * HW + e] = v0.y;
            s_tab[2 * HW + e] = v1.x, s_tab[3 * HW + e] = v1.y;
            s_tab[4 * HW + e] = v2.x, s_tab[5 * HW + e] = v2.y;
        }
        for (int e = threadIdx.x; e < TB * 6; e += TA) s_f[e] = (float)fk[(size_t)tB * TB * 6 + e];
        for (int e = threadIdx.x; e < TB; e += TA) s_off[e] = A.off_i[tB * TB + e];
        __syncthreads();
        const int base = (xa.x - ox) + A.W * (xa.y - oy);
#pragma unroll 8
        for (int j = 0; j < TB; j++) {
            const int idx = base - s_off[j];
            const float a11 = s_tab[idx], a12 = s_tab[HW + idx], a22 = s_tab[2 * HW + idx];
            const float a33 = s_tab[3 * HW + idx], b13 = s_tab[4 * HW + idx], b23 = s_tab[5 * HW + idx];
            const float* fj = s_f + j * 6;
            const float x0 = fj[0], x1 = fj[1], x2 = fj[2], y0 = fj[3], y1 = fj[4], y2 = fj[5];
            acc0 = fmaf(a11, x0, fmaf(a12, x1, fmaf(-b13, x2, acc0)));
            acc1 = fmaf(a12, x0, fmaf(a22, x1, fmaf(-b23, x2, acc1)));
            acc2 = fmaf(b13, x0, fmaf(b23, x1, fmaf(a33, x2, acc2)));
            acc3 = fmaf(a11, y0, fmaf(a12, y1, fmaf(-b13, y2, acc3)));
            acc4 = fmaf(a12, y0, fmaf(a22, y1, fmaf(-b23, y2, acc4)));
            acc5 = fmaf(b13, y0, fmaf(b23, y1, fmaf(a33, y2, acc5)));
        }
    }
    double* o = A.uh + (((size_t)r * A.K + k) * A.NPpad + a) * 6;
    o[0] = acc0, o[1] = acc1, o[2] = acc2, o[3] = acc3, o[4] = acc4, o[5] = acc5;
}


// FP32 with RB right-hand sides per thread: the staged table entries of a
// (pad column, interface column) pair are read once and applied to RB
// transformed force columns held in shared memory, so the gathers amortise
// over the right-hand sides and the loop is FFMA-bound.  grid.z = ceil(n_rhs / RB).
template <int TA, int TB, int RB>
__device__ __forceinline__ void tile_fp32_rb(const ContractArgs& A, int tA, int k, int rb, int n_rhs, void* smem_raw) {
    float* smem32rb = (float*)smem_raw;
    const int HW = A.H * A.W;
    float* s_tab = smem32rb;                          // [6][HW]
    // the force records start at the next 16-byte boundary after the table (HW may be odd)
    float4* s_fx = (float4*)((char*)smem32rb + (((size_t)6 * HW * 4 + 15) & ~(size_t)15));  // [RB][TB]: (x0, x1, x2, y0)
    float2* s_fy = (float2*)(s_fx + RB * TB);         // [RB][TB]: (y1, y2)
    int* s_off = (int*)(s_fy + RB * TB);              // [TB]
    const int r0 = rb * RB;
    const int a = tA * TA + threadIdx.x;
    const int2 xa = A.xy_p[a];
    const int4 bA = A.bbox_a[tA];
    float acc[RB][6];
#pragma unroll
    for (int q = 0; q < RB; q++)
#pragma unroll
        for (int c = 0; c < 6; c++) acc[q][c] = 0.f;
    const float* tk = A.tab32 + (size_t)(k - A.kbase) * A.Dy * A.Dx * 6;
    for (int tB = 0; tB < A.n_tb; tB++) {
        const int4 bB = A.bbox_b[tB];
        const int ox = bA.x - bB.y, oy = bA.z - bB.w;
        __syncthreads();
        for (int e = threadIdx.x; e < HW; e += TA) {
            const int iy = e / A.W, ix = e - iy * A.W;
            const int gx = ox + ix - A.box_x0, gy = oy + iy - A.box_y0;
            float2 v0 = make_float2(0, 0), v1 = v0, v2 = v0;
            if (gx < A.Dx && gy < A.Dy) {
                const float2* src = (const float2*)(tk + ((size_t)gy * A.Dx + gx) * 6);
                v0 = __ldg(src), v1 = __ldg(src + 1), v2 = __ldg(src + 2);
            }
            s_tab[0 * HW + e] = v0.x, s_tab[1 * HW + e] = v0.y;
            s_tab[2 * HW + e] = v1.x, s_tab[3 * HW + e] = v1.y;
            s_tab[4 * HW + e] = v2.x, s_tab[5 * HW + e] = v2.y;
        }
        for (int e = threadIdx.x; e < RB * TB; e += TA) {
            const int q = e / TB, j = e - q * TB;
            float v[6] = {0, 0, 0, 0, 0, 0};
            if (r0 + q < n_rhs) {
                const double* src = A.fh + (((size_t)(r0 + q) * A.K + k) * A.NIpad + (size_t)tB * TB + j) * 6;
#pragma unroll
                for (int c = 0; c < 6; c++) v[c] = (float)src[c];
            }
            s_fx[e] = make_float4(v[0], v[1], v[2], v[3]);
            s_fy[e] = make_float2(v[4], v[5]);
        }
        for (int e = threadIdx.x; e < TB; e += TA) s_off[e] = A.off_i[tB * TB + e];
        __syncthreads();
        const int base = (xa.x - ox) + A.W * (xa.y - oy);
#pragma unroll 2
        for (int j = 0; j < TB; j++) {
            const int idx = base - s_off[j];
            const float a11 = s_tab[idx], a12 = s_tab[HW + idx], a22 = s_tab[2 * HW + idx];
            const float a33 = s_tab[3 * HW + idx], b13 = s_tab[4 * HW + idx], b23 = s_tab[5 * HW + idx];
#pragma unroll
            for (int q = 0; q < RB; q++) {
                const float4 fx = s_fx[q * TB + j];
                const float2 fy = s_fy[q * TB + j];
                float* c = acc[q];
                c[0] = fmaf(a11, fx.x, fmaf(a12, fx.y, fmaf(-b13, fx.z, c[0])));
                c[1] = fmaf(a12, fx.x, fmaf(a22, fx.y, fmaf(-b23, fx.z, c[1])));
                c[2] = fmaf(b13, fx.x, fmaf(b23, fx.y, fmaf(a33, fx.z, c[2])));
                c[3] = fmaf(a11, fx.w, fmaf(a12, fy.x, fmaf(-b13, fy.y, c[3])));
                c[4] = fmaf(a12, fx.w, fmaf(a22, fy.x, fmaf(-b23, fy.y, c[4])));
                c[5] = fmaf(b13, fx.w, fmaf(b23, fy.x, fmaf(a33, fy.y, c[5])));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RB; q++) {
        if (r0 + q >= n_rhs) break;
        double* o = A.uh + (((size_t)(r0 + q) * A.K + k) * A.NPpad + a) * 6;
#pragma unroll
        for (int c = 0; c < 6; c++) o[c] = acc[q][c];
    }
}

// ---- double-float helpers -------------------------------------------------
struct df {
    float hi, lo;
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Accumulate the product (ah + al)(xh + xl) into the running pair (S, E),
// 10 FP32-pipe instructions.  The leading product p = fl(ah xh) is added to
// S as in Knuth's two-sum: s = S + p, bb = s - S is the part of p that s
// took up and S - (s - bb) the part of S it lost (exact).  What is left of
// the exact product, ah xh - bb, comes from one FMA (a single rounding of a
// quantity of order ulp(s)); it replaces both the two-sum's p - bb and the
// product's own rounding error ah xh - p.  The cross terms ah xl + al xh
// (relative size 2^-24) are added to it with two more FMAs, and everything
// low-order lands in E.
__device__ __forceinline__ void df_mac(float ah, float al, float xh, float xl, float& S, float& E) {
    const float p = __fmul_rn(ah, xh);
    const float s = __fadd_rn(S, p);
    const float bb = __fsub_rn(s, S);
    const float lost = __fsub_rn(S, __fsub_rn(s, bb));
    float rest = __fmaf_rn(ah, xh, -bb);
    rest = __fmaf_rn(ah, xl, rest);
    rest = __fmaf_rn(al, xh, rest);
    S = s;
    E = __fadd_rn(E, __fadd_rn(lost, rest));
}

// T += (S + E) in double-float arithmetic (accurate sum of two pairs).
__device__ __forceinline__ void df_fold(float& Thi, float& Tlo, float S, float E) {
    float s, e;
    two_sum(Thi, S, s, e);
    e = __fadd_rn(e, __fadd_rn(Tlo, E));
    Thi = __fadd_rn(s, e);
    Tlo = __fsub_rn(e, __fsub_rn(Thi, s));
}

// Double-float sub-box staging.  The table holds each entry as three 16-byte
// records (a11h, a11l, a12h, a12l), (a22h, a22l, a33h, a33l), (b13h, b13l,
// b23h, b23l), the layout kept in shared memory, so the W x H sub-box of a
// tile pair is a box of a three-dimensional tensor of 8-byte elements (6 Dx
// per table row, Dy rows, modes): H lines of 48 W contiguous bytes.  With a
// tensor map (tmap != nullptr) thread 0 fetches it with one TMA copy that
// completes on the barrier `bar` and zero-fills the part outside the table;
// without one (the persistent batch kernel, or a box line over the copy
// engine's 256 elements, W > 42) the CTA's threads copy it entry by entry.
__device__ __forceinline__ void x2_box_issue(const ContractArgs& A, int k, int ox, int oy, float4* s_tab,
                                             const void* tmap, uint64_t* bar, int nthreads) {
    if (tmap) {
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // after the last tile's reads
            tc::mbar_expect_tx(bar, (uint32_t)(A.H * A.W) * 48u);
            tc::tma_load_3d(s_tab, tmap, bar, 6 * (ox - A.box_x0), oy - A.box_y0, k - A.kbase);
        }
        return;
    }
    const float* tk = A.tabx2 + (size_t)(k - A.kbase) * A.Dy * A.Dx * 12;
    const int HW = A.H * A.W;
    for (int e = threadIdx.x; e < HW; e += nthreads) {
        const int iy = e / A.W, ix = e - iy * A.W;
        const int gx = ox + ix - A.box_x0, gy = oy + iy - A.box_y0;
        float4 q0 = make_float4(0, 0, 0, 0), q1 = q0, q2 = q0;
        if (gx < A.Dx && gy < A.Dy) {
            const float4* src = (const float4*)(tk + ((size_t)gy * A.Dx + gx) * 12);
            q0 = __ldg(src), q1 = __ldg(src + 1), q2 = __ldg(src + 2);
        }
        s_tab[3 * e] = q0, s_tab[3 * e + 1] = q1, s_tab[3 * e + 2] = q2;
    }
}

// The barrier before a tile's products.  With TMA staging every thread first
// waits (bounded) for the sub-box of interface tile tB, the barrier's phase
// tB.  Returns true for every thread of the CTA when a wait gave up: the CTA
// has then recorded the status word and waited once more (bounded) for its
// copy in flight, and leaves the tile without writing results.
__device__ __forceinline__ bool x2_box_wait(const ContractArgs& A, const void* tmap, uint64_t* bar, int tB) {
    if (!tmap) {
        __syncthreads();
        return false;
    }
    const bool late = !tc::mbar_wait(bar, (uint32_t)tB & 1u);
    if (!__syncthreads_or(late)) return false;
    if (threadIdx.x == 0) atomicExch(A.status, FBC_ERR_TIMEOUT);
    if (late) tc::mbar_wait(bar, (uint32_t)tB & 1u);
    return true;
}

// Double-float: the table sub-box staged as above and each interface column as
// four records: the (hi, lo) pairs of x and y' and off_b.
// K0: the tile of the one-mode k = 0 launches (a separate instance, so that the
// all-modes loop keeps its own code).
template <int TA, int TB, bool K0>
__device__ __forceinline__ void tile_x2(const ContractArgs& A, int tA, int k, int r, void* smem_raw,
                                        const void* tmap = nullptr, uint64_t* bar = nullptr) {
    float4* smemx2 = (float4*)smem_raw;
    const int HW = A.H * A.W;
    float4* s_tab = smemx2;            // [HW][3]
    float4* s_f = s_tab + 3 * HW;      // [TB][4]
    const int a = tA * TA + threadIdx.x;
    const int2 xa = A.xy_p[a];
    const int4 bA = A.bbox_a[tA];
    float Th[6] = {0, 0, 0, 0, 0, 0}, Tl[6] = {0, 0, 0, 0, 0, 0};
    const double* fk = A.fh + ((size_t)r * A.K + k) * A.NIpad * 6;
    for (int tB = 0; tB < A.n_tb; tB++) {
        const int4 bB = A.bbox_b[tB];
        const int ox = bA.x - bB.y, oy = bA.z - bB.w;
        __syncthreads();
        x2_box_issue(A, k, ox, oy, s_tab, tmap, bar, TA);
        for (int j = threadIdx.x; j < TB; j += TA) {
            float h[6], l[6];
#pragma unroll
            for (int c = 0; c < 6; c++) {
                const double v = fk[(size_t)(tB * TB + j) * 6 + c];
                h[c] = (float)v;
                l[c] = (float)(v - (double)h[c]);
            }
            s_f[4 * j + 0] = make_float4(h[0], l[0], h[1], l[1]);
            s_f[4 * j + 1] = make_float4(h[2], l[2], h[3], l[3]);
            s_f[4 * j + 2] = make_float4(h[4], l[4], h[5], l[5]);
            s_f[4 * j + 3] = make_float4(__int_as_float(A.off_i[tB * TB + j]), 0.f, 0.f, 0.f);
        }
        if (x2_box_wait(A, tmap, bar, tB)) return;
        const int base = (xa.x - ox) + A.W * (xa.y - oy);
        float S[6] = {0, 0, 0, 0, 0, 0}, E[6] = {0, 0, 0, 0, 0, 0};
        if (K0) {
            // k = 0: g^0 is real (B13 = B23 = 0) and so are the k = 0 forces, so of the
            // six outputs only x_0, x_1 and y'_2 are non-zero: 5 of the 18 products, in the
            // order the general loop adds them (the imaginary slots, which the inverse
            // transform discards at k = 0, are written as zeros below)
#pragma unroll 4
            for (int j = 0; j < TB; j++) {
                const float4 f0 = s_f[4 * j], f2 = s_f[4 * j + 2], f3 = s_f[4 * j + 3];
                const int idx = base - __float_as_int(f3.x);
                const float4 t0 = s_tab[3 * idx], t1 = s_tab[3 * idx + 1];
                df_mac(t0.x, t0.y, f0.x, f0.y, S[0], E[0]);
                df_mac(t0.z, t0.w, f0.z, f0.w, S[0], E[0]);
                df_mac(t0.z, t0.w, f0.x, f0.y, S[1], E[1]);
                df_mac(t1.x, t1.y, f0.z, f0.w, S[1], E[1]);
                df_mac(t1.z, t1.w, f2.z, f2.w, S[5], E[5]);
            }
#pragma unroll
            for (int c = 0; c < 6; c++) df_fold(Th[c], Tl[c], S[c], E[c]);
            continue;
        }
#pragma unroll 2
        for (int j = 0; j < TB; j++) {
            const float4 f0 = s_f[4 * j], f1 = s_f[4 * j + 1], f2 = s_f[4 * j + 2], f3 = s_f[4 * j + 3];
            const int idx = base - __float_as_int(f3.x);
            const float4 t0 = s_tab[3 * idx], t1 = s_tab[3 * idx + 1], t2 = s_tab[3 * idx + 2];
            // x = (f0.x, f0.y) (f0.z, f0.w) (f1.x, f1.y); y' = (f1.z, f1.w) (f2.x, f2.y) (f2.z, f2.w)
            df_mac(t0.x, t0.y, f0.x, f0.y, S[0], E[0]);
            df_mac(t0.z, t0.w, f0.z, f0.w, S[0], E[0]);
            df_mac(-t2.x, -t2.y, f1.x, f1.y, S[0], E[0]);
            df_mac(t0.z, t0.w, f0.x, f0.y, S[1], E[1]);
            df_mac(t1.x, t1.y, f0.z, f0.w, S[1], E[1]);
            df_mac(-t2.z, -t2.w, f1.x, f1.y, S[1], E[1]);
            df_mac(t2.x, t2.y, f0.x, f0.y, S[2], E[2]);
            df_mac(t2.z, t2.w, f0.z, f0.w, S[2], E[2]);
            df_mac(t1.z, t1.w, f1.x, f1.y, S[2], E[2]);
            df_mac(t0.x, t0.y, f1.z, f1.w, S[3], E[3]);
            df_mac(t0.z, t0.w, f2.x, f2.y, S[3], E[3]);
            df_mac(-t2.x, -t2.y, f2.z, f2.w, S[3], E[3]);
            df_mac(t0.z, t0.w, f1.z, f1.w, S[4], E[4]);
            df_mac(t1.x, t1.y, f2.x, f2.y, S[4], E[4]);
            df_mac(-t2.z, -t2.w, f2.z, f2.w, S[4], E[4]);
            df_mac(t2.x, t2.y, f1.z, f1.w, S[5], E[5]);
            df_mac(t2.z, t2.w, f2.x, f2.y, S[5], E[5]);
            df_mac(t1.z, t1.w, f2.z, f2.w, S[5], E[5]);
        }
#pragma unroll
        for (int c = 0; c < 6; c++) df_fold(Th[c], Tl[c], S[c], E[c]);
    }
    double* o = A.uh + (((size_t)r * A.K + k) * A.NPpad + a) * 6;
#pragma unroll
    for (int c = 0; c < 6; c++) o[c] = (double)Th[c] + (double)Tl[c];
    if (K0) o[2] = o[3] = o[4] = 0.0;
}


// Double-float for plans with several right-hand sides.  The CTA has NG
// groups of TA threads (thread = pad column a of the tile, group g) and covers
// NG * RB right-hand sides; thread (a, g) carries RB of them.  The staged
// table sub-box is shared by all groups, the three table records of a
// (pad column, interface column) pair are read once per thread and applied to
// its RB force columns, and each thread carries 6 RB independent running pairs
// (S, E): independent work for the FP32 pipes between the dependent adds of
// the two-sums.  The sums, their order and the fold per interface tile are
// those of tile_x2, so each right-hand side gets the same bits as from the
// one-rhs tile.  grid.z = ceil(n_rhs / (NG RB)); force records [NG RB][TB][3]
// (hi/lo pairs of x and y').
template <int TA, int TB, int NG, int RB, bool K0>
__device__ __forceinline__ void tile_x2_rb(const ContractArgs& A, int tA, int k, int rb, int n_rhs, void* smem_raw,
                                           const void* tmap, uint64_t* bar) {
    constexpr int NT = TA * NG, NR = NG * RB;
    float4* smemx2 = (float4*)smem_raw;
    const int HW = A.H * A.W;
    float4* s_tab = smemx2;                   // [HW][3]
    float4* s_f = s_tab + 3 * HW;             // [NR][TB][3]
    int* s_off = (int*)(s_f + 3 * NR * TB);   // [TB]
    const int r0 = rb * NR;
    const int a_loc = threadIdx.x % TA, g = threadIdx.x / TA;
    const int a = tA * TA + a_loc;
    const int2 xa = A.xy_p[a];
    const int4 bA = A.bbox_a[tA];
    float Th[RB][6], Tl[RB][6];
#pragma unroll
    for (int q = 0; q < RB; q++)
#pragma unroll
        for (int c = 0; c < 6; c++) Th[q][c] = Tl[q][c] = 0.f;
    for (int tB = 0; tB < A.n_tb; tB++) {
        const int4 bB = A.bbox_b[tB];
        const int ox = bA.x - bB.y, oy = bA.z - bB.w;
        __syncthreads();
        x2_box_issue(A, k, ox, oy, s_tab, tmap, bar, NT);
        for (int e = threadIdx.x; e < NR * TB; e += NT) {
            const int q = e / TB, j = e - q * TB;
            float h[6] = {0, 0, 0, 0, 0, 0}, l[6] = {0, 0, 0, 0, 0, 0};
            if (r0 + q < n_rhs) {
                const double* src = A.fh + (((size_t)(r0 + q) * A.K + k) * A.NIpad + (size_t)tB * TB + j) * 6;
#pragma unroll
                for (int c = 0; c < 6; c++) {
                    const double v = src[c];
                    h[c] = (float)v;
                    l[c] = (float)(v - (double)h[c]);
                }
            }
            s_f[3 * e + 0] = make_float4(h[0], l[0], h[1], l[1]);
            s_f[3 * e + 1] = make_float4(h[2], l[2], h[3], l[3]);
            s_f[3 * e + 2] = make_float4(h[4], l[4], h[5], l[5]);
        }
        for (int e = threadIdx.x; e < TB; e += NT) s_off[e] = A.off_i[tB * TB + e];
        if (x2_box_wait(A, tmap, bar, tB)) return;
        const int base = (xa.x - ox) + A.W * (xa.y - oy);
        float S[RB][6], E[RB][6];
#pragma unroll
        for (int q = 0; q < RB; q++)
#pragma unroll
            for (int c = 0; c < 6; c++) S[q][c] = E[q][c] = 0.f;
        const float4* fg = s_f + 3 * (g * RB) * TB;  // this group's right-hand sides
#pragma unroll 2
        for (int j = 0; j < TB; j++) {
            const int idx = base - s_off[j];
            const float4 t0 = s_tab[3 * idx], t1 = s_tab[3 * idx + 1];
            const float4 t2 = K0 ? make_float4(0, 0, 0, 0) : s_tab[3 * idx + 2];
#pragma unroll
            for (int q = 0; q < RB; q++) {
                const float4* fq = fg + 3 * (q * TB + j);
                const float4 f0 = fq[0], f2 = fq[2];
                if (K0) {
                    // k = 0: the five non-zero products of tile_x2's k = 0 branch, in its order
                    df_mac(t0.x, t0.y, f0.x, f0.y, S[q][0], E[q][0]);
                    df_mac(t0.z, t0.w, f0.z, f0.w, S[q][0], E[q][0]);
                    df_mac(t0.z, t0.w, f0.x, f0.y, S[q][1], E[q][1]);
                    df_mac(t1.x, t1.y, f0.z, f0.w, S[q][1], E[q][1]);
                    df_mac(t1.z, t1.w, f2.z, f2.w, S[q][5], E[q][5]);
                    continue;
                }
                const float4 f1 = fq[1];
                // x = (f0.x, f0.y) (f0.z, f0.w) (f1.x, f1.y); y' = (f1.z, f1.w) (f2.x, f2.y) (f2.z, f2.w)
                df_mac(t0.x, t0.y, f0.x, f0.y, S[q][0], E[q][0]);
                df_mac(t0.z, t0.w, f0.z, f0.w, S[q][0], E[q][0]);
                df_mac(-t2.x, -t2.y, f1.x, f1.y, S[q][0], E[q][0]);
                df_mac(t0.z, t0.w, f0.x, f0.y, S[q][1], E[q][1]);
                df_mac(t1.x, t1.y, f0.z, f0.w, S[q][1], E[q][1]);
                df_mac(-t2.z, -t2.w, f1.x, f1.y, S[q][1], E[q][1]);
                df_mac(t2.x, t2.y, f0.x, f0.y, S[q][2], E[q][2]);
                df_mac(t2.z, t2.w, f0.z, f0.w, S[q][2], E[q][2]);
                df_mac(t1.z, t1.w, f1.x, f1.y, S[q][2], E[q][2]);
                df_mac(t0.x, t0.y, f1.z, f1.w, S[q][3], E[q][3]);
                df_mac(t0.z, t0.w, f2.x, f2.y, S[q][3], E[q][3]);
                df_mac(-t2.x, -t2.y, f2.z, f2.w, S[q][3], E[q][3]);
                df_mac(t0.z, t0.w, f1.z, f1.w, S[q][4], E[q][4]);
                df_mac(t1.x, t1.y, f2.x, f2.y, S[q][4], E[q][4]);
                df_mac(-t2.z, -t2.w, f2.z, f2.w, S[q][4], E[q][4]);
                df_mac(t2.x, t2.y, f1.z, f1.w, S[q][5], E[q][5]);
                df_mac(t2.z, t2.w, f2.x, f2.y, S[q][5], E[q][5]);
                df_mac(t1.z, t1.w, f2.z, f2.w, S[q][5], E[q][5]);
            }
        }
#pragma unroll
        for (int q = 0; q < RB; q++)
#pragma unroll
            for (int c = 0; c < 6; c++) df_fold(Th[q][c], Tl[q][c], S[q][c], E[q][c]);
    }
#pragma unroll
    for (int q = 0; q < RB; q++) {
        const int r = r0 + g * RB + q;
        if (r >= n_rhs) break;
        double* o = A.uh + (((size_t)r * A.K + k) * A.NPpad + a) * 6;
#pragma unroll
        for (int c = 0; c < 6; c++) o[c] = (double)Th[q][c] + (double)Tl[q][c];
        if (K0) o[2] = o[3] = o[4] = 0.0;
    }
}


// ---- one launch per plan: grid (pad tiles, modes, right-hand sides) ----------
template <int TA, int TB>
__global__ void __launch_bounds__(TA) k_contract_fp64(ContractArgs A) {
    extern __shared__ float4 smem_raw[];
    tile_fp64<TA, TB>(A, blockIdx.x, A.k0 + blockIdx.y, blockIdx.z, smem_raw);
}
template <int TA, int TB>
__global__ void __launch_bounds__(TA) k_contract_fp32(ContractArgs A) {
    extern __shared__ float4 smem_raw[];
    tile_fp32<TA, TB>(A, blockIdx.x, A.k0 + blockIdx.y, blockIdx.z, smem_raw);
}
template <int TA, int TB, int RB>
__global__ void __launch_bounds__(TA) k_contract_fp32_rb(ContractArgs A, int n_rhs) {
    extern __shared__ float4 smem_raw[];
    tile_fp32_rb<TA, TB, RB>(A, blockIdx.x, A.k0 + blockIdx.y, blockIdx.z, n_rhs, smem_raw);
}
// The double-float kernels' shared memory: the sub-box at the first 128-byte boundary (the TMA
// destination's alignment; launches add 128 bytes), and the staging barrier, initialised by thread 0
// (the tile's first __syncthreads orders it before any use).  TMA: the sub-box comes by one tensor
// copy per tile (a compiled-in choice; the thread-staged instance serves boxes the copy cannot take).
__device__ __forceinline__ float4* x2_smem_setup(float4* smem_raw, uint64_t* bar, bool use_tma) {
    if (use_tma && threadIdx.x == 0) {
        tc::mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const uint32_t pad = (128u - (tc::smem_u32(smem_raw) & 127u)) & 127u;
    return (float4*)((char*)smem_raw + pad);
}
template <int TA, int TB, bool K0, bool TMA>
__global__ void __launch_bounds__(TA) k_contract_x2(ContractArgs A, const __grid_constant__ CUtensorMap tm) {
    extern __shared__ float4 smem_raw[];
    __shared__ uint64_t bar;
    float4* smem = x2_smem_setup(smem_raw, &bar, TMA);
    tile_x2<TA, TB, K0>(A, blockIdx.x, A.k0 + blockIdx.y, blockIdx.z, smem, TMA ? &tm : nullptr, &bar);
}
// grid (pad tiles, rhs groups, modes): the modes outermost, so the CTAs of all rhs groups of one mode run
// together and read that mode's table slice from L2
template <int TA, int TB, int NG, int RB, bool K0, bool TMA>
__global__ void __launch_bounds__(TA * NG) k_contract_x2_rb(ContractArgs A, const __grid_constant__ CUtensorMap tm,
                                                            int n_rhs) {
    extern __shared__ float4 smem_raw[];
    __shared__ uint64_t bar;
    float4* smem = x2_smem_setup(smem_raw, &bar, TMA);
    tile_x2_rb<TA, TB, NG, RB, K0>(A, blockIdx.x, A.k0 + blockIdx.z, blockIdx.y, n_rhs, smem, TMA ? &tm : nullptr,
                                   &bar);
}

// ---- batched: one persistent launch drains a cost-sorted work list ----------
// Item (inst, k, pad tile, r): r is a right-hand side, or a block of RB
// right-hand sides for the multi-rhs FP32 tile (k >= 1).  CTAs take items
// from a global counter with atomicAdd; no CTA ever waits for another.
constexpr int kBatchRB = 8;
template <int TA, int TB, int PREC, int PHASE>
__global__ void __launch_bounds__(TA) k_batch_contract(const ContractArgs* __restrict__ args,
                                                       const int* __restrict__ n_rhs_arr,
                                                       const int4* __restrict__ items, int n_items,
                                                       int* __restrict__ counter) {
    extern __shared__ float4 smem_raw[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();  // everyone has read s_item and left the previous tile's shared memory
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) return;
        const int4 w = items[it];
        const ContractArgs A = args[w.x];
        if (PREC == FBC_PREC_FP64) {
            tile_fp64<TA, TB>(A, w.z, w.y, w.w, smem_raw);
        } else if (PREC == FBC_PREC_F32X2) {
            tile_x2<TA, TB, false>(A, w.z, w.y, w.w, smem_raw);
        } else if (PHASE == 0) {
            tile_x2<TA, TB, true>(A, w.z, w.y, w.w, smem_raw);  // the k = 0 items
        } else {
            tile_fp32_rb<TA, TB, kBatchRB>(A, w.z, w.y, w.w, n_rhs_arr[w.x], smem_raw);
        }
    }
}

// multi-rhs double-float tile: kX2NG groups of kTileA threads, kX2RB right-hand sides per thread
constexpr int kX2NG = 2, kX2RB = 2, kX2R = kX2NG * kX2RB;
size_t x2_rb_smem(const Plan& P) {
    return (size_t)P.H * P.W * 48 + (size_t)kX2R * kTileB * 48 + (size_t)kTileB * 4 + 16 + 128;
}
size_t x2_smem(const Plan& P) { return (size_t)P.H * P.W * 48 + (size_t)kTileB * 64 + 16 + 128; }

// cuTensorMapEncodeTiled, reached through the runtime (no link against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn() {
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return (EncodeTiledFn)p;
    }();
    return fn;
}

// Tensor map of the double-float table for the TMA staging of a tile pair's sub-box: 8-byte
// elements in three dimensions (6 Dx per table row, Dy rows, n_slices mode slices), box (6 W, H, 1),
// zero outside the table.  A box starts at x = 6 (ox - box_x0): 48 bytes per entry, so on a
// 16-byte boundary.  Returns 0 (thread staging) when a box line is over the copy engine's 256
// elements (W > 42), H > 256, or the map cannot be made.
int encode_x2_map(const ContractArgs& A, int n_slices, CUtensorMap* m) {
    const EncodeTiledFn fn = encode_tiled_fn();
    if (!fn || !A.tabx2 || 6 * A.W > 256 || A.H > 256 || ((uintptr_t)A.tabx2 & 15u)) return 0;
    const cuuint64_t dims[3] = {6ull * A.Dx, (cuuint64_t)A.Dy, (cuuint64_t)n_slices};
    const cuuint64_t strides[2] = {48ull * A.Dx, 48ull * A.Dx * A.Dy};
    const cuuint32_t box[3] = {6u * (cuuint32_t)A.W, (cuuint32_t)A.H, 1};
    const cuuint32_t unit[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, (void*)A.tabx2, dims, strides, box, unit,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class T>
size_t contract_smem(const Plan& P, int TB, int per_entry) {
    return (size_t)6 * P.H * P.W * per_entry + (size_t)TB * 6 * per_entry + (size_t)TB * sizeof(int) + 16;
}

template <typename KernelT, typename... Extra>
cudaError_t launch_one(KernelT kern, const ContractArgs& A, dim3 grid, int threads, size_t smem, cudaStream_t st,
                       Extra... extra) {
    if (smem > 32 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e) return e;
    }
    kern<<<grid, threads, smem, st>>>(A, extra...);
    return cudaGetLastError();
}

// The double-float contraction of every mode (n_modes = K) or of the k = 0 mode alone (n_modes = 0:
// the one-mode instances).  Both tiles take the sub-box by TMA where the map can be made (measured
// faster than thread staging in each); otherwise the thread-staged instances run.
template <bool K0, bool TMA>
cudaError_t launch_x2_instance(Plan& P, const ContractArgs& A, int n_modes, int n_rhs, const CUtensorMap& tm,
                               cudaStream_t st) {
    if (n_rhs >= 2) {
        return launch_one(k_contract_x2_rb<kTileA, kTileB, kX2NG, kX2RB, K0, TMA>, A,
                          dim3(P.n_ta, (n_rhs + kX2R - 1) / kX2R, n_modes), kTileA * kX2NG, x2_rb_smem(P), st, tm,
                          n_rhs);
    }
    return launch_one(k_contract_x2<kTileA, kTileB, K0, TMA>, A, dim3(P.n_ta, n_modes, n_rhs), kTileA, x2_smem(P), st,
                      tm);
}
cudaError_t launch_contract_x2(Plan& P, const ContractArgs& A, int n_modes, int n_rhs, cudaStream_t st) {
    CUtensorMap tm{};
    const bool tma = encode_x2_map(A, A.tabx2 == P.d_table_x2 ? P.K : 1, &tm);
    if (n_modes == 0)
        return tma ? launch_x2_instance<true, true>(P, A, 1, n_rhs, tm, st)
                   : launch_x2_instance<true, false>(P, A, 1, n_rhs, tm, st);
    return tma ? launch_x2_instance<false, true>(P, A, n_modes, n_rhs, tm, st)
               : launch_x2_instance<false, false>(P, A, n_modes, n_rhs, tm, st);
}

}  // namespace

cudaError_t launch_contract(Plan& P, int n_rhs, cudaStream_t st) {
    static_assert(kTileA == 128 && kTileB == 64, "tile sizes are compiled in");
    ContractArgs A = make_contract_args(P);
    const size_t s64 = contract_smem<double>(P, kTileB, 8);
    if (s64 > 220 * 1024) return cudaErrorInvalidConfiguration;
    if (P.precision == FBC_PREC_FP64) {
        return launch_one(k_contract_fp64<kTileA, kTileB>, A, dim3(P.n_ta, P.K, n_rhs), kTileA, s64, st);
    }
    if (P.precision == FBC_PREC_FP32) {
        // logarithmic k = 0 mode in double-float (FP64-accurate), the rest in FP32
        cudaError_t e = launch_contract_x2_k0(P, A, n_rhs, st);
        if (e || P.K < 2) return e;
        A.k0 = 1;
        if (n_rhs >= 2) {
            constexpr int RB = 8;
            const size_t srb = (size_t)6 * P.H * P.W * 4 + (size_t)RB * kTileB * 24 + (size_t)kTileB * 4 + 16;
            return launch_one(k_contract_fp32_rb<kTileA, kTileB, RB>, A, dim3(P.n_ta, P.K - 1, (n_rhs + RB - 1) / RB),
                              kTileA, srb, st, n_rhs);
        }
        return launch_one(k_contract_fp32<kTileA, kTileB>, A, dim3(P.n_ta, P.K - 1, n_rhs), kTileA,
                          contract_smem<float>(P, kTileB, 4), st);
    }
    if (is_tensor_precision(P.precision)) {
        // logarithmic k = 0 mode in double-float (FP64-accurate) on the CUDA cores, k >= 1 on the tensor cores
        cudaError_t e = launch_contract_x2_k0(P, A, n_rhs, st);
        if (e || P.K < 2) return e;
        A.k0 = 1;
        return launch_contract_tc(A, P, n_rhs, st);
    }
    if (P.precision == FBC_PREC_F32X2) return launch_contract_x2(P, A, P.K, n_rhs, st);
    if (P.precision == FBC_PREC_BF16X6) {
        // k = 0 in double-float, k >= 1 in fixed-point slices on the tensor cores
        cudaError_t e = launch_contract_x2_k0(P, A, n_rhs, st);
        if (e || P.K < 2) return e;
        A.k0 = 1;
        return launch_contract_oz(A, P, n_rhs, st);
    }
    if (is_fft_precision(P.precision)) return launch_contract_fft(P, n_rhs, st);
    return cudaErrorInvalidValue;
}

ContractArgs make_contract_args(const Plan& P) {
    ContractArgs A;
    A.tab = P.d_table, A.tab32 = P.d_table32;
    // the double-float kernel of an FP32 or tensor-core plan only reads k = 0: the k = 0 slice suffices
    A.tabx2 = P.d_table_x2 ? P.d_table_x2 : P.d_table_x2_k0;
    A.fh = P.d_fh, A.uh = P.d_uh, A.uh32 = P.d_uh32, A.xy_p = P.d_xy_p, A.off_i = P.d_off_i;
    A.bbox_a = P.d_bbox_a, A.bbox_b = P.d_bbox_b;
    A.n_tb = P.n_tb, A.K = P.K, A.Dx = P.Dx, A.Dy = P.Dy, A.box_x0 = P.box_x0, A.box_y0 = P.box_y0;
    A.W = P.W, A.H = P.H, A.NIpad = P.NIpad, A.NPpad = P.NPpad, A.k0 = 0, A.kbase = 0;
    A.status = P.d_status;
    return A;
}

cudaError_t launch_contract_x2_k0(Plan& P, const ContractArgs& A, int n_rhs, cudaStream_t st) {
    return launch_contract_x2(P, A, 0, n_rhs, st);
}

cudaError_t launch_contract_modes(Plan& P, const ContractArgs& A0, int k0, int n_modes, int n_rhs, cudaStream_t st) {
    ContractArgs A = A0;
    A.k0 = k0;
    if (is_tensor_precision(P.precision)) return launch_contract_tc(A, P, n_rhs, st, n_modes);
    if (P.precision == FBC_PREC_FP32) {
        if (n_rhs >= 2) {
            constexpr int RB = 8;
            const size_t srb = (size_t)6 * P.H * P.W * 4 + (size_t)RB * kTileB * 24 + (size_t)kTileB * 4 + 16;
            return launch_one(k_contract_fp32_rb<kTileA, kTileB, RB>, A, dim3(P.n_ta, n_modes, (n_rhs + RB - 1) / RB),
                              kTileA, srb, st, n_rhs);
        }
        return launch_one(k_contract_fp32<kTileA, kTileB>, A, dim3(P.n_ta, n_modes, n_rhs), kTileA,
                          contract_smem<float>(P, kTileB, 4), st);
    }
    return cudaErrorInvalidValue;
}

size_t batch_contract_smem_phase(int precision, int phase, int W, int H) {
    const size_t HW = (size_t)W * H;
    const size_t s64 = HW * 48 + (size_t)kTileB * 52 + 16;
    const size_t sx2 = HW * 48 + (size_t)kTileB * 64 + 16;
    const size_t srb = ((HW * 24 + 15) & ~(size_t)15) + (size_t)kBatchRB * kTileB * 24 + (size_t)kTileB * 4 + 16;
    if (precision == FBC_PREC_FP64) return s64;
    if (precision == FBC_PREC_F32X2 || phase == 0) return sx2;
    return srb;
}

int batch_rhs_block() { return kBatchRB; }

template <int PREC, int PHASE>
static cudaError_t go_batch(const ContractArgs* d_args, const int* d_n_rhs, const int4* d_items, int n_items,
                            int* d_counter, int grid, size_t smem, cudaStream_t st) {
    auto kern = k_batch_contract<kTileA, kTileB, PREC, PHASE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    kern<<<grid, kTileA, smem, st>>>(d_args, d_n_rhs, d_items, n_items, d_counter);
    return cudaGetLastError();
}

template <int PREC, int PHASE>
static int occ_batch(size_t smem) {
    auto kern = k_batch_contract<kTileA, kTileB, PREC, PHASE>;
    int nb = 0;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kTileA, smem);
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

cudaError_t launch_batch_contract(int precision, int phase, const ContractArgs* d_args, const int* d_n_rhs,
                                  const int4* d_items, int n_items, int* d_counter, int grid, size_t smem,
                                  cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    if (precision == FBC_PREC_FP64) return go_batch<FBC_PREC_FP64, 1>(d_args, d_n_rhs, d_items, n_items, d_counter, grid, smem, st);
    if (precision == FBC_PREC_F32X2) return go_batch<FBC_PREC_F32X2, 1>(d_args, d_n_rhs, d_items, n_items, d_counter, grid, smem, st);
    if (phase == 0) return go_batch<FBC_PREC_FP32, 0>(d_args, d_n_rhs, d_items, n_items, d_counter, grid, smem, st);
    return go_batch<FBC_PREC_FP32, 1>(d_args, d_n_rhs, d_items, n_items, d_counter, grid, smem, st);
}

int batch_contract_occupancy_phase(int precision, int phase, size_t smem) {
    if (precision == FBC_PREC_FP64) return occ_batch<FBC_PREC_FP64, 1>(smem);
    if (precision == FBC_PREC_F32X2) return occ_batch<FBC_PREC_F32X2, 1>(smem);
    if (phase == 0) return occ_batch<FBC_PREC_FP32, 0>(smem);
    return occ_batch<FBC_PREC_FP32, 1>(smem);
}

}  // namespace fbc
