// H-matrix form of the pad update (Sec. 3.2; App., the construction of the H-matrix approximation of
// the Green matrix): the comparison form that the paper uses in place of the dense Green matrix.
//
// The Green matrix G~^{p|i+} has one row per pad atom (a, p) and component, and one column per
// interface atom (b, q) and component.  Its 3 x 3 blocks are G~(x_a - x_b, (p - q) c), the same
// periodic kernel (Sec. 3.1, Eqs. 32-36) that the per-mode forms transform along the line.
//
// Construction, in the paper's three steps:
//   Step 1 (host): cluster trees of the pad and interface atoms by geometric bisection.  A cluster of
//          more than b_min atoms is split at the midpoint of the longest side of its bounding box.
//          Atoms on the midpoint go to the first child, and both children keep the atoms' order.
//   Step 2 (host): the block partition.  t x s is admissible when min(diam t, diam s') <= gamma
//          dist(t, s') for s' in {s, s+, s-}: s and its images one period L c up and down, diam the
//          bounding-box diagonal, dist the centroid distance.  Admissible blocks are low-rank leaves,
//          inadmissible pairs of leaves are dense, and the rest are split.  Both steps use the same
//          double-precision operations in the same order as the test oracle, so the block lists
//          agree bit for bit.
//   Step 3 (device): adaptive cross approximation with partial pivoting, on atoms.  For the pivot
//          row atom the three residual rows are computed.  The column atom with the largest 3 x 3
//          residual block is chosen and its three residual columns computed.  Up to three rank-1
//          terms are taken from that 3 x 3 block by elimination with full pivoting; a pivot below
//          1e-6 of the block's first pivot ends the step.  The step's terms are then written as combinations of
//          the raw rows and columns.  A block stops after three consecutive steps whose terms have
//          Frobenius norm <= eps ||S||_F.  ||S||_F is kept exactly with the cross terms
//          2 sum_{l,m} (u_l . u_m)(v_l . v_m).  The next pivot atom is the unused row atom where the
//          new columns are largest.
//          All blocks of a wave iterate in lockstep.  One iteration is nine launches over the wave's
//          (block, chunk) items: residual rows, pivot column, residual columns, 3 x 3 elimination,
//          emission of the terms (row and column halves), dot products with the earlier terms (row
//          and column halves), and the stopping test.  The work of a step is O(k (n_t + n_s)) and
//          is spread over the whole GPU whatever the blocks' sizes.  Entries come from the plan's
//          periodic kernel, evaluated once in real space and stored as an FP32 box table.  The
//          terms are stored in FP32, but the residual entries G - sum_l u_l v_l are summed in
//          double-float: the terms of a cross approximation cancel strongly, and plain FP32 sums
//          leave a noise floor near 5e-5 that the approximation then fits (measured: 5.4e-5 on
//          the small ring at eps = 1e-5, against 6e-6 with FP64 arithmetic).  The running norms
//          are FP64; the paper's eps = 1e-5 is inside the range accepted (eps >= 1e-6).
// Apply, u <- beta u + alpha G_H (f - mean f):
//   gather: f in cluster order, FP32, after the neutral projection;
//   z_b = V_b^T x_s for every low-rank block (items of 256 column dofs, then a fixed-order sum);
//   one CTA per row leaf: y = sum over the blocks that cover the leaf's rows of U_b z_b (and
//   D_b x_s for dense blocks), in the blocks' order.  Warps own rows and sums are FP64, so the result
//   is deterministic.  The epilogue writes u in the caller's layout; an optional zero mean follows.
//   For the same cancellation, z and U_b z_b are summed in double-float (z kept as an FP32 pair).
// Storage for the apply is FP32: U_b [3 n_t][k] and V_b [3 n_s][k], row-major (a row's k
// coefficients contiguous), and D_b [3 n_t][3 n_s].  The apply reads each factor once per group
// of up to four right-hand sides.

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "fbc_internal.cuh"

namespace {

constexpr float kPivotDrop = 1e-6f;  // a pivot below this fraction of the block's first ends a step
constexpr int kStopSteps = 3;        // consecutive small steps that stop a block
constexpr int kChunk = 256;          // atoms per CTA item of the build (rows or columns)
constexpr int kDotChunk = 4096;      // dofs per CTA item of the dot products
constexpr int kRG = 4;               // right-hand sides per pass of the apply
constexpr int kZCols = 256;          // column dofs per item of z = V^T x
constexpr int kMaxRank = 6141;       // the build's slots (rank + 3) stay <= 6144
constexpr int kDefaultMaxRank = kMaxRank;
constexpr size_t kBuildSmemMax = sizeof(float) * 3 * (kMaxRank + 3);  // k_aca_rows / k_aca_cols

// ------------------------------------------------------------------------------------- host side

struct Tree {
    std::vector<int64_t> perm;  // cluster order position -> atom id (column * L + repeat)
    std::vector<int64_t> start, count;
    std::vector<std::array<int64_t, 3>> lo, hi, sum;
    std::vector<int32_t> kid0, kid1;  // -1 for a leaf
    double c = 1.0;
    bool leaf(int n) const { return kid0[n] < 0; }
    void centroid(int n, double out[3]) const {
        const double k = (double)count[n];
        out[0] = (double)sum[n][0] / k;
        out[1] = (double)sum[n][1] / k;
        out[2] = ((double)sum[n][2] / k) * c;
    }
    double diam2(int n) const {
        const double dx = (double)(hi[n][0] - lo[n][0]);
        const double dy = (double)(hi[n][1] - lo[n][1]);
        const double dz = (double)(hi[n][2] - lo[n][2]) * c;
        return (dx * dx + dy * dy) + dz * dz;
    }
};

struct TreeBuilder {
    const std::vector<std::array<int64_t, 3>>& pts;
    Tree& T;
    int b_min;
    int build(int64_t start, int64_t count) {
        const int me = (int)T.start.size();
        std::array<int64_t, 3> lo = pts[T.perm[start]], hi = lo, sm = {0, 0, 0};
        for (int64_t k = start; k < start + count; k++) {
            const auto& p = pts[T.perm[k]];
            for (int a = 0; a < 3; a++) {
                lo[a] = std::min(lo[a], p[a]);
                hi[a] = std::max(hi[a], p[a]);
                sm[a] += p[a];
            }
        }
        T.start.push_back(start);
        T.count.push_back(count);
        T.lo.push_back(lo);
        T.hi.push_back(hi);
        T.sum.push_back(sm);
        T.kid0.push_back(-1);
        T.kid1.push_back(-1);
        if (count > b_min) {
            const double ext[3] = {(double)(hi[0] - lo[0]), (double)(hi[1] - lo[1]), (double)(hi[2] - lo[2]) * T.c};
            int ax = 0;
            for (int a = 1; a < 3; a++)
                if (ext[a] > ext[ax]) ax = a;  // the first longest side
            const int64_t two_mid = lo[ax] + hi[ax];
            auto first = T.perm.begin() + start;
            auto mid = std::stable_partition(first, first + count,
                                             [&](int64_t id) { return 2 * pts[id][ax] <= two_mid; });
            const int64_t n1 = mid - first;
            if (n1 > 0 && n1 < count) {
                const int a = build(start, n1);
                const int b = build(start + n1, count - n1);
                T.kid0[me] = a;
                T.kid1[me] = b;
            }
        }
        return me;
    }
};

void build_tree(const int32_t* xy, int n, int L, double c, int b_min, Tree& T) {
    std::vector<std::array<int64_t, 3>> pts((size_t)n * L);
    for (int a = 0; a < n; a++)
        for (int p = 0; p < L; p++) pts[(size_t)a * L + p] = {xy[2 * a], xy[2 * a + 1], p};
    T = Tree();
    T.c = c;
    T.perm.resize(pts.size());
    std::iota(T.perm.begin(), T.perm.end(), 0);
    TreeBuilder tb{pts, T, b_min};
    tb.build(0, (int64_t)pts.size());
}

bool admissible(const Tree& Tt, int t, const Tree& Ts, int s, double gamma, double period) {
    double ct[3], cs[3];
    Tt.centroid(t, ct);
    Ts.centroid(s, cs);
    const double m = std::min(Tt.diam2(t), Ts.diam2(s));
    const double g2 = gamma * gamma;
    const double shifts[3] = {0.0, period, -period};
    for (double sh : shifts) {
        const double dx = ct[0] - cs[0];
        const double dy = ct[1] - cs[1];
        const double dz = ct[2] - (cs[2] + sh);
        if (!(m <= g2 * ((dx * dx + dy * dy) + dz * dz))) return false;
    }
    return true;
}

struct BlockRec {
    int64_t r0, nr, c0, nc, lowrank;
    bool operator<(const BlockRec& o) const {
        if (r0 != o.r0) return r0 < o.r0;
        if (nr != o.nr) return nr < o.nr;
        if (c0 != o.c0) return c0 < o.c0;
        if (nc != o.nc) return nc < o.nc;
        return lowrank < o.lowrank;
    }
};

void partition(const Tree& Tp, const Tree& Ti, double gamma, double period, std::vector<BlockRec>& out) {
    out.clear();
    std::vector<std::pair<int, int>> stack{{0, 0}};
    while (!stack.empty()) {
        const auto [t, s] = stack.back();
        stack.pop_back();
        if (admissible(Tp, t, Ti, s, gamma, period)) {
            out.push_back({Tp.start[t], Tp.count[t], Ti.start[s], Ti.count[s], 1});
            continue;
        }
        const bool lt = Tp.leaf(t), ls = Ti.leaf(s);
        if (lt && ls) {
            out.push_back({Tp.start[t], Tp.count[t], Ti.start[s], Ti.count[s], 0});
            continue;
        }
        const int ta[2] = {lt ? t : Tp.kid0[t], lt ? -1 : Tp.kid1[t]};
        const int sa[2] = {ls ? s : Ti.kid0[s], ls ? -1 : Ti.kid1[s]};
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++)
                if (ta[i] >= 0 && sa[j] >= 0) stack.push_back({ta[i], sa[j]});
    }
    std::sort(out.begin(), out.end());
}

int check_partition_args(const int32_t* xy_i, int32_t n_i, const int32_t* xy_p, int32_t n_p, int32_t L, double c,
                         double gamma, int32_t b_min) {
    if (!xy_i || !xy_p || n_i < 1 || n_p < 1 || L < 1) return fbc::report_error(FBC_ERR_INVALID_ARG, "bad geometry");
    if (!(c > 0.0) || !std::isfinite(c)) return fbc::report_error(FBC_ERR_INVALID_ARG, "c must be positive");
    if (!(gamma > 0.0) || !std::isfinite(gamma)) return fbc::report_error(FBC_ERR_INVALID_ARG, "gamma must be positive");
    if (b_min < 1) return fbc::report_error(FBC_ERR_INVALID_ARG, "b_min must be >= 1");
    if ((int64_t)n_i * L > (int64_t)1 << 30 || (int64_t)n_p * L > (int64_t)1 << 30)
        return fbc::report_error(FBC_ERR_INVALID_ARG, "too many atoms");
    return FBC_OK;
}

// ------------------------------------------------------------------------------------- device side

struct Geom {
    const int4* ra;    // [n_p L] pad atoms in cluster order: (x, y, p, 0)
    const int4* ca;    // [n_i L] interface atoms in cluster order: (x, y, q, 0)
    const float* tab;  // [Dy Dx][L/2 + 1][6] real-space kernel
    int Dx, box_x0, box_y0, L, Lh;
};

// The 3 x 3 block G~(x_a - x_b, (p - q) c), row-major.
__device__ __forceinline__ void entry9(const Geom& g, int4 a, int4 b, float G[9]) {
    const long long cell = (long long)(a.y - b.y - g.box_y0) * g.Dx + (a.x - b.x - g.box_x0);
    int s = a.z - b.z;
    if (s < 0) s += g.L;
    float sg = 1.0f;
    if (s > g.Lh) {  // G~(d, -s) = M G~(d, s) M with M = diag(1, 1, -1)
        s = g.L - s;
        sg = -1.0f;
    }
    const float2* t = reinterpret_cast<const float2*>(g.tab + (cell * (g.Lh + 1) + s) * 6);
    const float2 t01 = __ldg(t), t23 = __ldg(t + 1), t45 = __ldg(t + 2);
    G[0] = t01.x, G[1] = t01.y, G[2] = sg * t45.x;
    G[3] = t01.y, G[4] = t23.x, G[5] = sg * t45.y;
    G[6] = sg * t45.x, G[7] = sg * t45.y, G[8] = t23.y;
}

struct BuildBlk {     // one low-rank block of a wave
    int r0, nr, c0, nc;  // atoms, cluster order
    long long offU;      // U slots: scratch[offU + slot * 3 nr + i]
    long long offV;      // V slots: scratch[offV + slot * 3 nc + j]
    long long offDU;     // dot partials of the row items: [item][3][kcap]
    long long offDV;     // dot partials of the column items
    long long used;      // first word of the used-row bitmap
    int kcap;            // a block stops once it has this many terms (min(full, max_rank))
    int slots;           // kcap + 3: a step starts below kcap and adds at most 3 terms
    int full;            // min(3 nr, 3 nc): a factorisation of this rank is exact
    int it_r0, n_it_r;   // row items (kChunk atoms) of this block in the wave's row list
    int it_c0, n_it_c;   // column items
    int dt_r0, n_dt_r;   // dot items over rows (kDotChunk dofs)
    int dt_c0, n_dt_c;   // dot items over columns
};

struct BuildState {
    int k;         // terms so far
    int ia;        // pivot row atom (block-local)
    int ja;        // pivot column atom
    int m;         // terms of this step
    int active;    // 1 while the block iterates
    int skip;      // this step found no nonzero residual: nothing to emit
    int small;     // consecutive small steps
    int capped;    // stopped at kcap before the rule held
    double S2;     // ||S||_F^2
    double p0;     // the block's first pivot (0 until the first step): the scale of the drop rule
    float P[9];    // the 3 x 3 residual pivot block
    // the step's elimination, replayed by the emit kernel on every row and column:
    // u_q = C'_{pb[q]} / piv[q], v_q = R'_{pa[q]}; then C'_b -= u_q rowv[q][b], R'_a -= colv[q][a] v_q
    int pa[3], pb[3];
    float piv[3];
    float rowv[9];  // P'_q[pa[q]][b]: v_q at the pivot column atom's columns
    float colv[9];  // P'_q[a][pb[q]] / piv[q]: u_q at the pivot row atom's rows
};

// (S, E) <- (S, E) + a b, a double-float sum of FP32 products: Knuth's two-sum on S, and the
// product's own rounding error carried by one FMA (a b - bb is formed exactly and rounded once).
// The terms of a cross approximation cancel strongly (their sum is far smaller than the largest
// term), so plain FP32 sums of them lose the accuracy that eps asks for.  The round-to-nearest
// intrinsics keep the compiler from fusing a b + S into one FMA, which would break the two-sum.
__device__ __forceinline__ void df_mac(float& S, float& E, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float s = __fadd_rn(S, p);
    const float bb = __fsub_rn(s, S);
    const float lost = __fsub_rn(S, __fsub_rn(s, bb));
    const float rest = __fmaf_rn(a, b, -bb);
    S = s;
    E = __fadd_rn(E, __fadd_rn(lost, rest));
}

// (S, E) <- (S, E) + (S2, E2): two-sum of the leading parts, the rest added to the trailing part.
__device__ __forceinline__ void df_add(float& S, float& E, float S2, float E2) {
    const float s = __fadd_rn(S, S2);
    const float bb = __fsub_rn(s, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(S2, bb));
    E = __fadd_rn(__fadd_rn(E, E2), err);
    S = s;
}

// The warp's double-float sum, in FP32 operations (no FP64 pipe work per row); every lane gets it.
__device__ __forceinline__ void df_warp_sum(float& S, float& E) {
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, S, o), e2 = __shfl_xor_sync(0xffffffffu, E, o);
        df_add(S, E, s2, e2);
    }
}

__device__ __forceinline__ void argmax_merge(float& v, int& i, float v2, int i2) {
    if (v2 > v || (v2 == v && i2 < i)) v = v2, i = i2;
}

// Block-wide (max value, lowest index) over 256 threads.
__device__ __forceinline__ void block_argmax(float& v, int& i) {
    __shared__ float sv[8];
    __shared__ int si[8];
    for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        argmax_merge(v, i, v2, i2);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sv[w] = v, si[w] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) argmax_merge(v, i, sv[k], si[k]);
    }
}

// Step (a): the residual rows R_i = G[(ia, i), :] - sum_l U_l[(ia, i)] V_l, written to V slots k..k+2,
// and per item the column atom with the largest 3 x 3 residual block.
__global__ void __launch_bounds__(256) k_aca_rows(const BuildBlk* __restrict__ B, const BuildState* __restrict__ S,
                                                   const int2* __restrict__ items, Geom g, float* __restrict__ w,
                                                   float2* __restrict__ pmax) {
    extern __shared__ float su[];  // [k][3]
    const int2 it = items[blockIdx.x];
    const BuildBlk b = B[it.x];
    const BuildState& st = S[it.x];
    if (!st.active) return;
    const int k = st.k, ia = st.ia;
    const long long nr3 = 3LL * b.nr, nc3 = 3LL * b.nc;
    const float* U = w + b.offU;
    float* V = w + b.offV;
    for (int t = threadIdx.x; t < 3 * k; t += blockDim.x) su[t] = U[(t / 3) * nr3 + 3 * ia + t % 3];
    __syncthreads();
    const int ca = it.y + threadIdx.x;
    float best = -1.0f;
    int barg = 0x7fffffff;
    if (ca < b.nc) {
        float acc[9], err[9];
        entry9(g, g.ra[b.r0 + ia], g.ca[b.c0 + ca], acc);
#pragma unroll
        for (int t = 0; t < 9; t++) err[t] = 0.0f;
        const float* v = V + 3LL * ca;
        for (int l = 0; l < k; l++, v += nc3) {
            const float v0 = v[0], v1 = v[1], v2 = v[2];
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const float u = -su[3 * l + i];
                df_mac(acc[3 * i + 0], err[3 * i + 0], u, v0);
                df_mac(acc[3 * i + 1], err[3 * i + 1], u, v1);
                df_mac(acc[3 * i + 2], err[3 * i + 2], u, v2);
            }
        }
#pragma unroll
        for (int t = 0; t < 9; t++) acc[t] += err[t];
        float n2 = 0.0f;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int jj = 0; jj < 3; jj++) {
                V[(long long)(k + i) * nc3 + 3LL * ca + jj] = acc[3 * i + jj];
                n2 = fmaf(acc[3 * i + jj], acc[3 * i + jj], n2);
            }
        best = n2, barg = ca;
    }
    block_argmax(best, barg);
    if (threadIdx.x == 0) pmax[blockIdx.x] = make_float2(best, __int_as_float(barg));
}

// Step (b), one warp per block: the pivot column atom, the 3 x 3 pivot block; the pivot row is used.
__global__ void k_aca_pick(const BuildBlk* __restrict__ B, BuildState* __restrict__ S, const float2* __restrict__ pmax,
                           unsigned* __restrict__ used, const float* __restrict__ w, int* __restrict__ n_active) {
    const int bi = blockIdx.x, lane = threadIdx.x;
    BuildState& st = S[bi];
    if (!st.active) return;
    const BuildBlk b = B[bi];
    float best = -1.0f;
    int barg = 0x7fffffff;
    for (int t = lane; t < b.n_it_c; t += 32) {
        const float2 p = pmax[b.it_c0 + t];
        argmax_merge(best, barg, p.x, __float_as_int(p.y));
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, barg, o);
        argmax_merge(best, barg, v2, i2);
    }
    unsigned* bits = used + b.used;
    if (lane == 0) bits[st.ia >> 5] |= 1u << (st.ia & 31);
    __syncwarp();
    if (best > 0.0f) {
        if (lane < 9) {
            const long long nc3 = 3LL * b.nc;
            st.P[lane] = w[b.offV + (long long)(st.k + lane / 3) * nc3 + 3LL * barg + lane % 3];
        }
        if (lane == 0) st.ja = barg, st.skip = 0;
        return;
    }
    // the residual of this row atom vanishes: take the first unused row atom, if any
    const int nwords = (b.nr + 31) >> 5;
    int next = 0x7fffffff;
    for (int wd = lane; wd < nwords; wd += 32) {
        unsigned free_bits = ~bits[wd];
        if (wd == nwords - 1 && (b.nr & 31)) free_bits &= (1u << (b.nr & 31)) - 1u;
        if (free_bits) {
            next = min(next, wd * 32 + __ffs(free_bits) - 1);
            break;
        }
    }
    for (int o = 16; o > 0; o >>= 1) next = min(next, __shfl_xor_sync(0xffffffffu, next, o));
    if (lane == 0) {
        st.skip = 1;
        if (next == 0x7fffffff) {
            st.active = 0;
            atomicSub(n_active, 1);
        } else {
            st.ia = next;
        }
    }
}

// Step (c): the residual columns C_jj = G[:, (ja, jj)] - sum_l V_l[(ja, jj)] U_l, written to U slots k..k+2.
__global__ void __launch_bounds__(256) k_aca_cols(const BuildBlk* __restrict__ B, const BuildState* __restrict__ S,
                                                   const int2* __restrict__ items, Geom g, float* __restrict__ w) {
    extern __shared__ float sv[];  // [k][3]
    const int2 it = items[blockIdx.x];
    const BuildBlk b = B[it.x];
    const BuildState& st = S[it.x];
    if (!st.active || st.skip) return;
    const int k = st.k, ja = st.ja;
    const long long nr3 = 3LL * b.nr, nc3 = 3LL * b.nc;
    float* U = w + b.offU;
    const float* V = w + b.offV;
    for (int t = threadIdx.x; t < 3 * k; t += blockDim.x) sv[t] = V[(t / 3) * nc3 + 3 * ja + t % 3];
    __syncthreads();
    const int ra = it.y + threadIdx.x;
    if (ra >= b.nr) return;
    float acc[9], err[9];
    entry9(g, g.ra[b.r0 + ra], g.ca[b.c0 + ja], acc);
#pragma unroll
    for (int t = 0; t < 9; t++) err[t] = 0.0f;
    const float* u = U + 3LL * ra;
    for (int l = 0; l < k; l++, u += nr3) {
        const float u0 = -u[0], u1 = -u[1], u2 = -u[2];
#pragma unroll
        for (int jj = 0; jj < 3; jj++) {
            const float v = sv[3 * l + jj];
            df_mac(acc[0 + jj], err[0 + jj], u0, v);
            df_mac(acc[3 + jj], err[3 + jj], u1, v);
            df_mac(acc[6 + jj], err[6 + jj], u2, v);
        }
    }
#pragma unroll
    for (int t = 0; t < 9; t++) acc[t] += err[t];
#pragma unroll
    for (int ii = 0; ii < 3; ii++)
#pragma unroll
        for (int jj = 0; jj < 3; jj++) U[(long long)(k + jj) * nr3 + 3LL * ra + ii] = acc[3 * ii + jj];
}

// Step (d), one thread per block: elimination with full pivoting on the 3 x 3 pivot block (FP64 from
// the FP32 block).  The pivot sequence and the factors that update the other rows and columns are
// kept for the emit kernel, which repeats the same elimination on every row and column of the block.
__global__ void k_aca_pivot(BuildState* __restrict__ S, int n) {
    const int bi = blockIdx.x * blockDim.x + threadIdx.x;
    if (bi >= n) return;
    BuildState& st = S[bi];
    if (!st.active || st.skip) return;
    double P[9];
    for (int t = 0; t < 9; t++) P[t] = st.P[t];
    double p0 = st.p0;
    int m = 0;
    for (int step = 0; step < 3; step++) {
        int a = 0, bcol = 0;
        double amax = -1.0;
        for (int t = 0; t < 9; t++)
            if (fabs(P[t]) > amax) amax = fabs(P[t]), a = t / 3, bcol = t % 3;
        const double piv = P[3 * a + bcol];
        if (p0 == 0.0) p0 = fabs(piv);
        // pivots at the rounding level that the FP32 terms leave in the residual (about 6e-8 of
        // the block's scale) would add noise and could fill a small block's rank
        if (!(fabs(piv) > (double)kPivotDrop * p0)) break;
        st.pa[m] = a, st.pb[m] = bcol, st.piv[m] = (float)piv;
        for (int t = 0; t < 3; t++) {
            st.rowv[3 * m + t] = (float)P[3 * a + t];
            st.colv[3 * m + t] = (float)(P[3 * t + bcol] / piv);
        }
        m++;
        double Po[9];
        for (int t = 0; t < 9; t++) Po[t] = P[t];
        for (int a2 = 0; a2 < 3; a2++)
            for (int b2 = 0; b2 < 3; b2++) P[3 * a2 + b2] = Po[3 * a2 + b2] - Po[3 * a2 + bcol] * Po[3 * a + b2] / piv;
    }
    st.p0 = p0;
    st.m = m;
}

// Step (e): the step's terms from the raw rows and columns, in place in slots k..k+m-1, by the pivot
// kernel's elimination repeated on each atom's rows (or columns) in FP32.  Row items
// also give the Gram partials of the new u and the unused row atom where they are largest; column
// items give the Gram partials of the new v.
template <bool ROWS>
__global__ void __launch_bounds__(256) k_aca_emit(const BuildBlk* __restrict__ B, const BuildState* __restrict__ S,
                                                   const int2* __restrict__ items, const unsigned* __restrict__ used,
                                                   float* __restrict__ w, double* __restrict__ gram,
                                                   float2* __restrict__ rmax) {
    const int2 it = items[blockIdx.x];
    const BuildBlk b = B[it.x];
    const BuildState& st = S[it.x];
    if (!st.active || st.skip) return;
    const int k = st.k, m = st.m;
    const int n = ROWS ? b.nr : b.nc;
    const long long n3 = 3LL * n;
    float* X = w + (ROWS ? b.offU : b.offV);
    const int at = it.y + threadIdx.x;
    double g6[6] = {0, 0, 0, 0, 0, 0};
    float best = -1.0f;
    int barg = 0x7fffffff;
    if (at < n) {
        float raw[3][3], out[3][3];  // raw[s][e]: raw column (rows) or row (columns) s at dof e
#pragma unroll
        for (int s2 = 0; s2 < 3; s2++)
#pragma unroll
            for (int e = 0; e < 3; e++) raw[s2][e] = X[(long long)(k + s2) * n3 + 3LL * at + e];
#pragma unroll
        for (int q = 0; q < 3; q++) {
#pragma unroll
            for (int e = 0; e < 3; e++) out[q][e] = 0.0f;
            if (q < m) {
                if (ROWS) {  // u_q = C'_b / piv, then C'_b2 -= u_q rowv[q][b2]
                    const int bq = st.pb[q];
                    const float pv = st.piv[q];
#pragma unroll
                    for (int e = 0; e < 3; e++) out[q][e] = (bq == 0 ? raw[0][e] : bq == 1 ? raw[1][e] : raw[2][e]) / pv;
#pragma unroll
                    for (int b2 = 0; b2 < 3; b2++)
#pragma unroll
                        for (int e = 0; e < 3; e++) raw[b2][e] = fmaf(-out[q][e], st.rowv[3 * q + b2], raw[b2][e]);
                } else {  // v_q = R'_a, then R'_a2 -= colv[q][a2] v_q
                    const int aq = st.pa[q];
#pragma unroll
                    for (int e = 0; e < 3; e++) out[q][e] = aq == 0 ? raw[0][e] : aq == 1 ? raw[1][e] : raw[2][e];
#pragma unroll
                    for (int a2 = 0; a2 < 3; a2++)
#pragma unroll
                        for (int e = 0; e < 3; e++) raw[a2][e] = fmaf(-st.colv[3 * q + a2], out[q][e], raw[a2][e]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 3; q++)
            if (q < m) {
#pragma unroll
                for (int e = 0; e < 3; e++) X[(long long)(k + q) * n3 + 3LL * at + e] = out[q][e];
            }
        int t = 0;
#pragma unroll
        for (int q = 0; q < 3; q++)
#pragma unroll
            for (int q2 = q; q2 < 3; q2++, t++)
                g6[t] = (double)out[q][0] * out[q2][0] + (double)out[q][1] * out[q2][1] + (double)out[q][2] * out[q2][2];
        if (ROWS) {
            const unsigned* bits = used + b.used;
            if (!((bits[at >> 5] >> (at & 31)) & 1u)) best = (float)(g6[0] + g6[3] + g6[5]), barg = at;
        }
    }
    __shared__ double sg[8][6];
    for (int t = 0; t < 6; t++) {
        double v = g6[t];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        g6[t] = v;
    }
    if ((threadIdx.x & 31) == 0)
        for (int t = 0; t < 6; t++) sg[threadIdx.x >> 5][t] = g6[t];
    if (ROWS) block_argmax(best, barg);
    else __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 0; t < 6; t++) {
            double v = 0.0;
            for (int ww = 0; ww < (int)(blockDim.x >> 5); ww++) v += sg[ww][t];
            gram[6LL * blockIdx.x + t] = v;
        }
        if (ROWS) rmax[blockIdx.x] = make_float2(best, __int_as_float(barg));
    }
}

// Step (f): partial dot products of the step's terms with the earlier ones over a chunk of dofs:
// part[item][q][l] = sum_{i in chunk} X_l[i] X_{k+q}[i], l < k.  Warps over l, lanes over dofs.  The
// terms of a cross approximation are much larger than their sum and cancel, so ||S||_F^2 built from
// plain FP32 dot products drifts by more than S itself (it went negative on a 720 x 480-atom block,
// and the stopping rule then never held): double-float per lane, FP64 across lanes and chunks.
template <bool ROWS>
__global__ void __launch_bounds__(256) k_aca_dots(const BuildBlk* __restrict__ B, const BuildState* __restrict__ S,
                                                   const int2* __restrict__ items, const float* __restrict__ w,
                                                   double* __restrict__ part) {
    __shared__ float snew[3][kDotChunk];
    const int2 it = items[blockIdx.x];
    const BuildBlk b = B[it.x];
    const BuildState& st = S[it.x];
    if (!st.active || st.skip) return;
    const int k = st.k, m = st.m;
    const long long n3 = 3LL * (ROWS ? b.nr : b.nc);
    const float* X = w + (ROWS ? b.offU : b.offV);
    const long long i0 = (long long)it.y * kDotChunk;
    const int cnt = (int)min((long long)kDotChunk, n3 - i0);
    for (int q = 0; q < 3; q++)
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) snew[q][t] = q < m ? X[(long long)(k + q) * n3 + i0 + t] : 0.0f;
    __syncthreads();
    double* out = part + (ROWS ? b.offDU : b.offDV) + (long long)(it.y) * 3 * b.slots;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int l = warp; l < k; l += (int)(blockDim.x >> 5)) {
        const float* xl = X + (long long)l * n3 + i0;
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, e0 = 0.0f, e1 = 0.0f, e2 = 0.0f;
        for (int t = lane; t < cnt; t += 32) {
            const float x = xl[t];
            df_mac(s0, e0, x, snew[0][t]);
            df_mac(s1, e1, x, snew[1][t]);
            df_mac(s2, e2, x, snew[2][t]);
        }
        double a0 = (double)s0 + (double)e0, a1 = (double)s1 + (double)e1, a2 = (double)s2 + (double)e2;
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) out[l] = a0, out[b.slots + l] = a1, out[2 * b.slots + l] = a2;
    }
}

// Step (g), one CTA per block: ||S||_F^2 += 2 <S, dS> + ||dS||^2, the stopping rule, the next pivot row.
__global__ void __launch_bounds__(256) k_aca_finish(const BuildBlk* __restrict__ B, BuildState* __restrict__ S,
                                                     const double* __restrict__ part, const double* __restrict__ gram_r,
                                                     const double* __restrict__ gram_c, const float2* __restrict__ rmax,
                                                     double eps, int* __restrict__ n_active) {
    const BuildBlk b = B[blockIdx.x];
    BuildState& st = S[blockIdx.x];
    if (!st.active) return;
    if (st.skip) {  // the pick step already chose the next row
        __syncthreads();
        if (threadIdx.x == 0) st.skip = 0;
        return;
    }
    const int k = st.k, m = st.m;
    // <S, dS> = sum_l sum_q (U_l . u_q)(V_l . v_q)
    double cross = 0.0;
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
        for (int q = 0; q < m; q++) {
            double du = 0.0, dv = 0.0;
            for (int t = 0; t < b.n_dt_r; t++) du += part[b.offDU + (long long)t * 3 * b.slots + q * b.slots + l];
            for (int t = 0; t < b.n_dt_c; t++) dv += part[b.offDV + (long long)t * 3 * b.slots + q * b.slots + l];
            cross += du * dv;
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = cross;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    float best = -1.0f;
    int barg = 0x7fffffff;
    for (int t = threadIdx.x; t < b.n_it_r; t += blockDim.x) {
        const float2 p = rmax[b.it_r0 + t];
        argmax_merge(best, barg, p.x, __float_as_int(p.y));
    }
    block_argmax(best, barg);
    if (threadIdx.x == 0) {
        double gu[6] = {0, 0, 0, 0, 0, 0}, gv[6] = {0, 0, 0, 0, 0, 0};
        for (int t = 0; t < b.n_it_r; t++)
            for (int e = 0; e < 6; e++) gu[e] += gram_r[6LL * (b.it_r0 + t) + e];
        for (int t = 0; t < b.n_it_c; t++)
            for (int e = 0; e < 6; e++) gv[e] += gram_c[6LL * (b.it_c0 + t) + e];
        // ||dS||^2 = sum_{q,q2} (u_q . u_q2)(v_q . v_q2); the 6 entries are the upper triangle
        const double step2 = gu[0] * gv[0] + gu[3] * gv[3] + gu[5] * gv[5] +
                             2.0 * (gu[1] * gv[1] + gu[2] * gv[2] + gu[4] * gv[4]);
        st.S2 += 2.0 * red[0] + step2;
        st.k = k + m;
        const bool small = m == 0 || sqrt(fmax(step2, 0.0)) <= eps * sqrt(fmax(st.S2, 0.0));
        st.small = small ? st.small + 1 : 0;
        bool done = st.small >= kStopSteps || best < 0.0f;
        if (!done && st.k >= b.kcap) done = true, st.capped = b.kcap < b.full;
        if (done) {
            st.active = 0;
            atomicSub(n_active, 1);
        } else {
            st.ia = barg;
        }
    }
}

// The wave's factors in the apply layout: dst[i][l] = src[l][i] (i < n3, l < k).
__global__ void k_transpose(const float* __restrict__ src, float* __restrict__ dst, long long n3, int k) {
    __shared__ float tile[32][33];
    const long long i0 = (long long)blockIdx.x * 32;
    const int l0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int l = l0 + r;
        const long long i = i0 + threadIdx.x;
        tile[r][threadIdx.x] = (l < k && i < n3) ? src[(long long)l * n3 + i] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long i = i0 + r;
        const int l = l0 + threadIdx.x;
        if (i < n3 && l < k) dst[i * k + l] = tile[threadIdx.x][r];
    }
}

// Dense blocks: D[3 ra + ii][3 ca + jj], one thread per atom pair.
__global__ void k_dense_fill(Geom g, int r0, int nr, int c0, int nc, float* __restrict__ D) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nr * nc) return;
    const int ra = (int)(t / nc), ca = (int)(t % nc);
    float G[9];
    entry9(g, g.ra[r0 + ra], g.ca[c0 + ca], G);
    const long long nc3 = 3LL * nc;
    for (int ii = 0; ii < 3; ii++)
        for (int jj = 0; jj < 3; jj++) D[(3LL * ra + ii) * nc3 + 3LL * ca + jj] = G[3 * ii + jj];
}

// ------------------------------------------------------------------------------------- apply kernels

struct ApplyBlk {
    const float* U;  // [3 nr][k] (low rank) or D [3 nr][3 nc] (dense)
    const float* V;  // [3 nc][k] (low rank)
    int r0, nr, c0, nc, k, lowrank;
    long long offZ;  // z of the block: zbuf[offZ + r k + l]
    int zit0, n_zit; // its items of z = V^T x
};

// Per-chunk sums of f over interface atoms, per right-hand side and component (FP64).
__global__ void k_hm_fsum(const double* __restrict__ f, long long n_at, double* __restrict__ part) {
    const int r = blockIdx.y;
    double s[3] = {0.0, 0.0, 0.0};
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < n_at; a += (long long)gridDim.x * blockDim.x)
        for (int j = 0; j < 3; j++) s[j] += f[((long long)r * n_at + a) * 3 + j];
    __shared__ double red[3][256];
    for (int j = 0; j < 3; j++) red[j][threadIdx.x] = s[j];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int j = 0; j < 3; j++) red[j][threadIdx.x] += red[j][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[((long long)r * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = red[threadIdx.x][0];
}

// mean[r][j] = sum of the partials / n_at, in a fixed order.
__global__ void k_hm_mean(const double* __restrict__ part, int n_part, long long n_at, double* __restrict__ mean) {
    const int r = blockIdx.x, j = threadIdx.x;
    if (j >= 3) return;
    double s = 0.0;
    for (int t = 0; t < n_part; t++) s += part[((long long)r * n_part + t) * 3 + j];
    mean[3 * r + j] = s / (double)n_at;
}

// x[r][3 cpos + j] = f[r][atom(cpos)][j] - mean[r][j], FP32, cluster order.
__global__ void k_hm_gather(const double* __restrict__ f, const int* __restrict__ perm, long long n_at, int rg,
                            const double* __restrict__ mean, float* __restrict__ x) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)rg * n_at * 3) return;
    const int r = (int)(t / (n_at * 3));
    const long long rem = t - (long long)r * n_at * 3;
    const long long cpos = rem / 3;
    const int j = (int)(rem % 3);
    const double v = f[((long long)r * n_at + perm[cpos]) * 3 + j] - (mean ? mean[3 * r + j] : 0.0);
    x[t] = (float)v;
}

// z partials: for an item (block, 256 column dofs), zp[item][r][l] = sum_j V[j][l] x[r][c0 3 + j],
// summed in double-float and stored in FP64.
template <int RG>  // right-hand sides of this pass (1..kRG)
__global__ void __launch_bounds__(256) k_hm_z(const ApplyBlk* __restrict__ A, const int2* __restrict__ items,
                                               const float* __restrict__ x, long long ncol3,
                                               double* __restrict__ zp, const long long* __restrict__ zp_off) {
    constexpr int rg = RG;
    __shared__ float sx[kRG][kZCols];
    const int2 it = items[blockIdx.x];
    const ApplyBlk b = A[it.x];
    const long long j0 = (long long)it.y * kZCols;
    const int cnt = (int)min((long long)kZCols, 3LL * b.nc - j0);
    for (int t = threadIdx.x; t < kRG * kZCols; t += blockDim.x) {
        const int r = t / kZCols, j = t % kZCols;
        sx[r][j] = (j < cnt && r < rg) ? x[(long long)r * ncol3 + 3LL * b.c0 + j0 + j] : 0.0f;
    }
    __syncthreads();
    double* out = zp + zp_off[blockIdx.x];
    const float* V = b.V + j0 * b.k;
    for (int l = threadIdx.x; l < b.k; l += blockDim.x) {
        // four interleaved chains over j (columns j = c mod 4), joined in a fixed order
        float acc[4][RG], err[4][RG];
#pragma unroll
        for (int c = 0; c < 4; c++)
#pragma unroll
            for (int r = 0; r < RG; r++) acc[c][r] = 0.0f, err[c][r] = 0.0f;
        const float* v = V + l;
        int j = 0;
        for (; j + 4 <= cnt; j += 4, v += 4LL * b.k) {
            float vv[4];
#pragma unroll
            for (int c = 0; c < 4; c++) vv[c] = v[(long long)c * b.k];
#pragma unroll
            for (int c = 0; c < 4; c++)
#pragma unroll
                for (int r = 0; r < RG; r++) df_mac(acc[c][r], err[c][r], vv[c], sx[r][j + c]);
        }
        for (int c = 0; j < cnt; j++, c++, v += b.k) {
            const float vv = *v;
#pragma unroll
            for (int r = 0; r < RG; r++) df_mac(acc[0][r], err[0][r], vv, sx[r][j]);
        }
#pragma unroll
        for (int r = 0; r < RG; r++) {
            df_add(acc[0][r], err[0][r], acc[1][r], err[1][r]);
            df_add(acc[2][r], err[2][r], acc[3][r], err[3][r]);
            df_add(acc[0][r], err[0][r], acc[2][r], err[2][r]);
            out[(long long)r * b.k + l] = (double)acc[0][r] + (double)err[0][r];
        }
    }
}

// z[b][r][l] = sum over the block's items of the partials, in a fixed order, kept as an FP32 pair
// (hi, lo) with hi + lo = z to about 48 bits.  CTA (b, tile): 32 entries t of z_b times 8 subsets
// of the items (item i in subset i mod 8); the subsets meet in order.  A block's items are
// consecutive in the partial buffer, kRG k numbers apart.
__global__ void __launch_bounds__(256) k_hm_zsum(const ApplyBlk* __restrict__ A, const double* __restrict__ zp,
                                                  const long long* __restrict__ zp_off, int rg, float2* __restrict__ z) {
    __shared__ double red[8][32];
    const ApplyBlk b = A[blockIdx.x];
    if (!b.lowrank || b.n_zit == 0) return;
    const int n = rg * b.k;
    const int t = blockIdx.y * 32 + (threadIdx.x & 31), sub = threadIdx.x >> 5;
    if (blockIdx.y * 32 >= n) return;
    const long long base = zp_off[b.zit0], stride = (long long)kRG * b.k;
    double c = 0.0;
    if (t < n)
        for (int i = sub; i < b.n_zit; i += 8) c += zp[base + (long long)i * stride + t];
    red[sub][threadIdx.x & 31] = c;
    __syncthreads();
    if (sub == 0 && t < n) {
        double s = 0.0;
        for (int q = 0; q < 8; q++) s += red[q][threadIdx.x];
        const float hi = (float)s;
        z[b.offZ + t] = make_float2(hi, (float)(s - (double)hi));
    }
}

// One CTA per row leaf: y = sum over the covering blocks of U z (or D x); then the epilogue
// u = beta u + alpha y in the caller's layout, and the leaf's sums of the new u (zero mean).
template <int RG>  // right-hand sides of this pass (1..kRG)
__global__ void __launch_bounds__(256) k_hm_y(const ApplyBlk* __restrict__ A, const int* __restrict__ leaf_r0,
                                               const int* __restrict__ leaf_nr, const int* __restrict__ cover_off,
                                               const int* __restrict__ cover, const float2* __restrict__ z,
                                               const float* __restrict__ x, long long ncol3, const int* __restrict__ perm_p,
                                               long long n_pat, double alpha, double beta,
                                               double* __restrict__ u, double* __restrict__ usum, int max_rows) {
    constexpr int rg = RG;
    extern __shared__ unsigned char smem_raw[];
    double* y = reinterpret_cast<double*>(smem_raw);  // [rows][kRG]
    const int lf = blockIdx.x;
    const int R0 = leaf_r0[lf], NR = leaf_nr[lf];
    const int rows = 3 * NR;
    for (int t = threadIdx.x; t < rows * kRG; t += blockDim.x) y[t] = 0.0;
    __syncthreads();  // from here on each row's sums belong to one warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = cover_off[lf]; c < cover_off[lf + 1]; c++) {
        const ApplyBlk b = A[cover[c]];
        const long long row0 = 3LL * (R0 - b.r0);  // the leaf's first row within the block
        if (b.lowrank) {
            const float2* zb = z + b.offZ;  // read by every row of the leaf: from L1
            constexpr int RR = 4;            // rows per warp at a time: each z load serves four rows
            for (int i0 = warp; i0 < rows; i0 += nw * RR) {
                float acc[RR][RG], err[RR][RG];
                const float* ur[RR];
#pragma unroll
                for (int q = 0; q < RR; q++) {
                    const int i = min(i0 + q * nw, rows - 1);  // rows past the leaf repeat its last row
                    ur[q] = b.U + (row0 + i) * b.k;
#pragma unroll
                    for (int r = 0; r < RG; r++) acc[q][r] = 0.0f, err[q][r] = 0.0f;
                }
                for (int l = lane; l < b.k; l += 32) {
                    float2 zz[RG];
#pragma unroll
                    for (int r = 0; r < RG; r++) zz[r] = __ldg(zb + r * b.k + l);
#pragma unroll
                    for (int q = 0; q < RR; q++) {
                        const float uv = ur[q][l];
#pragma unroll
                        for (int r = 0; r < RG; r++) {
                            df_mac(acc[q][r], err[q][r], uv, zz[r].x);
                            err[q][r] = __fmaf_rn(uv, zz[r].y, err[q][r]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < RR; q++) {
                    const int i = i0 + q * nw;
#pragma unroll
                    for (int r = 0; r < RG; r++) {
                        df_warp_sum(acc[q][r], err[q][r]);
                        if (lane == 0 && i < rows) y[i * kRG + r] += (double)acc[q][r] + (double)err[q][r];
                    }
                }
            }
        } else {
            const long long nc3 = 3LL * b.nc;
            for (int i = warp; i < rows; i += nw) {
                const float* dr = b.U + (row0 + i) * nc3;
                float acc[RG];
#pragma unroll
                for (int r = 0; r < RG; r++) acc[r] = 0.0f;
                for (long long j = lane; j < nc3; j += 32) {
                    const float dv = dr[j];
#pragma unroll
                    for (int r = 0; r < RG; r++) acc[r] = fmaf(dv, x[(long long)r * ncol3 + 3LL * b.c0 + j], acc[r]);
                }
#pragma unroll
                for (int r = 0; r < RG; r++)
                    for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
                if (lane == 0) {
#pragma unroll
                    for (int r = 0; r < RG; r++) y[i * kRG + r] += (double)acc[r];
                }
            }
        }
    }
    __syncthreads();
    // epilogue (the new u goes back into y); then the leaf's sums of the new u for the zero mean
    for (int t = threadIdx.x; t < rows * rg; t += blockDim.x) {
        const int i = t % rows, r = t / rows;
        const long long atom = perm_p[R0 + i / 3];
        const long long idx = ((long long)r * n_pat + atom) * 3 + i % 3;
        const double v = alpha * y[i * kRG + r] + (beta != 0.0 ? beta * u[idx] : 0.0);
        u[idx] = v;
        y[i * kRG + r] = v;
    }
    if (usum) {
        __shared__ double red[256];
        for (int r = 0; r < rg; r++)
            for (int j = 0; j < 3; j++) {
                __syncthreads();
                double v = 0.0;
                for (int i = j + 3 * (int)threadIdx.x; i < rows; i += 3 * (int)blockDim.x) v += y[i * kRG + r];
                red[threadIdx.x] = v;
                __syncthreads();
                for (int o = 128; o > 0; o >>= 1) {
                    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
                    __syncthreads();
                }
                if (threadIdx.x == 0) usum[((long long)r * gridDim.x + lf) * 3 + j] = red[0];
            }
    }
}

__global__ void k_hm_usub(double* __restrict__ u, long long n_pat, const double* __restrict__ mean) {
    const int r = blockIdx.y;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_pat * 3; t += (long long)gridDim.x * blockDim.x)
        u[(long long)r * n_pat * 3 + t] -= mean[3 * r + (int)(t % 3)];
}

}  // namespace

// ------------------------------------------------------------------------------------- the object

struct fbc_hmat {
    int device = 0;
    int n_i = 0, n_p = 0, L = 0;
    fbc_hmat_options opt{};
    fbc_hmat_info info{};
    std::vector<BlockRec> blocks;
    std::vector<int32_t> ranks;
    std::vector<std::pair<float*, float*>> factor_ptrs;  // (U, V) of a low-rank block; (D, null) of a dense one
    std::vector<void*> arenas;       // device allocations of the factors
    ApplyBlk* d_blocks = nullptr;    // [n_blocks]
    int n_leaves = 0, max_leaf_rows = 0, max_k = 0;
    int* d_leaf_r0 = nullptr;
    int* d_leaf_nr = nullptr;
    int* d_cover_off = nullptr;
    int* d_cover = nullptr;
    int* d_perm_i = nullptr;         // cluster order -> interface atom id
    int* d_perm_p = nullptr;         // cluster order -> pad atom id
    int2* d_zitems = nullptr;
    long long* d_zp_off = nullptr;
    int n_zitems = 0;
    float* d_x = nullptr;            // [kRG][3 n_i L]
    double* d_zp = nullptr;          // z partials per item (FP64)
    float2* d_z = nullptr;           // z of each low-rank block as (hi, lo)
    double* d_fpart = nullptr;       // [kRG][kFParts][3]
    double* d_mean = nullptr;        // [kRG][3]
    double* d_usum = nullptr;        // [kRG][n_leaves][3]
    size_t apply_smem = 0;
};

namespace {

constexpr int kFParts = 304;

void free_hmat(fbc_hmat* h) {
    for (void* a : h->arenas) cudaFree(a);
    void* bufs[] = {h->d_blocks, h->d_leaf_r0, h->d_leaf_nr, h->d_cover_off, h->d_cover, h->d_perm_i, h->d_perm_p,
                    h->d_zitems, h->d_zp_off, h->d_x, h->d_zp, h->d_z, h->d_fpart, h->d_mean, h->d_usum};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete h;
}

int hfail(int code, const char* msg) { return fbc::report_error(code, msg); }

int hcuda(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return fbc::report_error(e == cudaErrorMemoryAllocation ? FBC_ERR_OOM : FBC_ERR_CUDA, buf);
}

template <class T>
int halloc(T** p, size_t count, const char* what) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    const char* inj = getenv("FBC_TEST_FAIL_ALLOC");
    if (inj && strcmp(inj, what) == 0) {
        char buf[128];
        snprintf(buf, sizeof(buf), "injected allocation failure: %s", what);
        return hfail(FBC_ERR_OOM, buf);
    }
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return hcuda(e, what);
    }
    return FBC_OK;
}

#define HCHK(call)                                   \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return hcuda(e_, #call); \
    } while (0)

// Original column order from the plan's sorted layout.
void original_sites(const std::vector<int>& perm, const std::vector<int2>& sorted, int n, std::vector<int32_t>& xy) {
    xy.assign(2 * (size_t)n, 0);
    for (size_t s = 0; s < perm.size(); s++)
        if (perm[s] >= 0) xy[2 * perm[s]] = sorted[s].x, xy[2 * perm[s] + 1] = sorted[s].y;
}

// Step 3 for the low-rank blocks listed in `wave` (indices into h->blocks); their factors go to
// one new arena in the apply layout.
int build_wave(fbc_hmat* h, const std::vector<int>& wave, const Geom& g, cudaStream_t st) {
    const int nb = (int)wave.size();
    std::vector<BuildBlk> bb(nb);
    std::vector<int2> it_r, it_c, dt_r, dt_c;
    long long scratch = 0, dpart = 0, used_words = 0;
    int max_k = 0;
    for (int w = 0; w < nb; w++) {
        const BlockRec& r = h->blocks[wave[w]];
        BuildBlk& b = bb[w];
        b.r0 = (int)r.r0, b.nr = (int)r.nr, b.c0 = (int)r.c0, b.nc = (int)r.nc;
        b.full = (int)std::min(3 * r.nr, 3 * r.nc);
        b.kcap = std::min(b.full, h->opt.max_rank);
        b.slots = b.kcap + 3;
        const int slots = b.slots;
        b.offU = scratch;
        scratch += (long long)slots * 3 * b.nr;
        b.offV = scratch;
        scratch += (long long)slots * 3 * b.nc;
        scratch = (scratch + 31) & ~31LL;
        b.used = used_words;
        used_words += (b.nr + 31) / 32;
        b.it_r0 = (int)it_r.size();
        for (int a = 0; a < b.nr; a += kChunk) it_r.push_back(make_int2(w, a));
        b.n_it_r = (int)it_r.size() - b.it_r0;
        b.it_c0 = (int)it_c.size();
        for (int a = 0; a < b.nc; a += kChunk) it_c.push_back(make_int2(w, a));
        b.n_it_c = (int)it_c.size() - b.it_c0;
        b.dt_r0 = (int)dt_r.size();
        for (long long i = 0, c = 0; i < 3LL * b.nr; i += kDotChunk, c++) dt_r.push_back(make_int2(w, (int)c));
        b.n_dt_r = (int)dt_r.size() - b.dt_r0;
        b.dt_c0 = (int)dt_c.size();
        for (long long i = 0, c = 0; i < 3LL * b.nc; i += kDotChunk, c++) dt_c.push_back(make_int2(w, (int)c));
        b.n_dt_c = (int)dt_c.size() - b.dt_c0;
        b.offDU = dpart;
        dpart += (long long)b.n_dt_r * 3 * slots;
        b.offDV = dpart;
        dpart += (long long)b.n_dt_c * 3 * slots;
        max_k = std::max(max_k, slots);
    }
    float* d_w = nullptr;
    double* d_part = nullptr;
    double* d_gr = nullptr;
    double* d_gc = nullptr;
    float2* d_pmax = nullptr;
    float2* d_rmax = nullptr;
    unsigned* d_used = nullptr;
    BuildBlk* d_bb = nullptr;
    BuildState* d_st = nullptr;
    int2 *d_itr = nullptr, *d_itc = nullptr, *d_dtr = nullptr, *d_dtc = nullptr;
    int* d_nact = nullptr;
    int rc = FBC_OK;
    auto cleanup = [&]() {
        void* bufs[] = {d_w, d_part, d_gr, d_gc, d_pmax, d_rmax, d_used, d_bb, d_st, d_itr, d_itc, d_dtr, d_dtc, d_nact};
        for (void* p : bufs)
            if (p) cudaFree(p);
    };
#define WALLOC(p, n, what)                     \
    do {                                       \
        if ((rc = halloc(&(p), (n), what))) {  \
            cleanup();                         \
            return rc;                         \
        }                                      \
    } while (0)
#define WCHK(call)                         \
    do {                                   \
        cudaError_t e_ = (call);           \
        if (e_ != cudaSuccess) {           \
            rc = hcuda(e_, #call);         \
            cleanup();                     \
            return rc;                     \
        }                                  \
    } while (0)
    WALLOC(d_w, (size_t)scratch, "hmat_build_scratch");
    WALLOC(d_part, (size_t)std::max(dpart, 1LL), "hmat_build_dots");
    WALLOC(d_gr, 6 * it_r.size(), "hmat_build_gram");
    WALLOC(d_gc, 6 * it_c.size(), "hmat_build_gram");
    WALLOC(d_pmax, it_c.size(), "hmat_build_pivots");
    WALLOC(d_rmax, it_r.size(), "hmat_build_pivots");
    WALLOC(d_used, (size_t)used_words, "hmat_build_used");
    WALLOC(d_bb, (size_t)nb, "hmat_build_blocks");
    WALLOC(d_st, (size_t)nb, "hmat_build_blocks");
    WALLOC(d_itr, it_r.size(), "hmat_build_items");
    WALLOC(d_itc, it_c.size(), "hmat_build_items");
    WALLOC(d_dtr, dt_r.size(), "hmat_build_items");
    WALLOC(d_dtc, dt_c.size(), "hmat_build_items");
    WALLOC(d_nact, 1, "hmat_build_items");
    std::vector<BuildState> s0(nb);
    for (auto& s : s0) {
        memset(&s, 0, sizeof(s));
        s.active = 1;
    }
    WCHK(cudaMemcpyAsync(d_bb, bb.data(), sizeof(BuildBlk) * nb, cudaMemcpyHostToDevice, st));
    WCHK(cudaMemcpyAsync(d_st, s0.data(), sizeof(BuildState) * nb, cudaMemcpyHostToDevice, st));
    WCHK(cudaMemcpyAsync(d_itr, it_r.data(), sizeof(int2) * it_r.size(), cudaMemcpyHostToDevice, st));
    WCHK(cudaMemcpyAsync(d_itc, it_c.data(), sizeof(int2) * it_c.size(), cudaMemcpyHostToDevice, st));
    WCHK(cudaMemcpyAsync(d_dtr, dt_r.data(), sizeof(int2) * dt_r.size(), cudaMemcpyHostToDevice, st));
    WCHK(cudaMemcpyAsync(d_dtc, dt_c.data(), sizeof(int2) * dt_c.size(), cudaMemcpyHostToDevice, st));
    WCHK(cudaMemsetAsync(d_used, 0, sizeof(unsigned) * (size_t)used_words, st));
    WCHK(cudaMemcpyAsync(d_nact, &nb, sizeof(int), cudaMemcpyHostToDevice, st));
    // at most 3 x 6144 floats (kMaxRank + 3 slots); the kernels' limit is raised once per create
    const size_t smem_k = sizeof(float) * 3 * (size_t)max_k;
    // every iteration adds a term or uses up a row atom
    long long max_iter = 0;
    for (const auto& b : bb) max_iter = std::max<long long>(max_iter, (long long)b.slots + b.nr + 8);
    int n_act = nb;
    for (long long iter = 0; iter < max_iter && n_act > 0; iter++) {
        k_aca_rows<<<(unsigned)it_c.size(), 256, smem_k, st>>>(d_bb, d_st, d_itc, g, d_w, d_pmax);
        k_aca_pick<<<nb, 32, 0, st>>>(d_bb, d_st, d_pmax, d_used, d_w, d_nact);
        k_aca_cols<<<(unsigned)it_r.size(), 256, smem_k, st>>>(d_bb, d_st, d_itr, g, d_w);
        k_aca_pivot<<<(nb + 127) / 128, 128, 0, st>>>(d_st, nb);
        k_aca_emit<true><<<(unsigned)it_r.size(), 256, 0, st>>>(d_bb, d_st, d_itr, d_used, d_w, d_gr, d_rmax);
        k_aca_emit<false><<<(unsigned)it_c.size(), 256, 0, st>>>(d_bb, d_st, d_itc, d_used, d_w, d_gc, nullptr);
        k_aca_dots<true><<<(unsigned)dt_r.size(), 256, 0, st>>>(d_bb, d_st, d_dtr, d_w, d_part);
        k_aca_dots<false><<<(unsigned)dt_c.size(), 256, 0, st>>>(d_bb, d_st, d_dtc, d_w, d_part);
        k_aca_finish<<<nb, 256, 0, st>>>(d_bb, d_st, d_part, d_gr, d_gc, d_rmax, h->opt.eps, d_nact);
        WCHK(cudaGetLastError());
        if ((iter & 7) == 7) {
            WCHK(cudaMemcpyAsync(&n_act, d_nact, sizeof(int), cudaMemcpyDeviceToHost, st));
            WCHK(cudaStreamSynchronize(st));
        }
    }
    if (n_act > 0) {
        WCHK(cudaMemcpyAsync(&n_act, d_nact, sizeof(int), cudaMemcpyDeviceToHost, st));
        WCHK(cudaStreamSynchronize(st));
        if (n_act > 0) {
            cleanup();
            return hfail(FBC_ERR_CUDA, "H-matrix build: blocks still active after the iteration bound");
        }
    }
    std::vector<BuildState> sf(nb);
    WCHK(cudaMemcpyAsync(sf.data(), d_st, sizeof(BuildState) * nb, cudaMemcpyDeviceToHost, st));
    WCHK(cudaStreamSynchronize(st));
    size_t total = 0;
    for (int w = 0; w < nb; w++) total += (size_t)sf[w].k * 3 * (bb[w].nr + bb[w].nc);
    float* arena = nullptr;
    WALLOC(arena, std::max<size_t>(total, 1), "hmat_factors");
    h->arenas.push_back(arena);
    size_t off = 0;
    for (int w = 0; w < nb; w++) {
        const int k = sf[w].k;
        const int bi = wave[w];
        h->ranks[bi] = k;
        h->info.n_capped += sf[w].capped;
        float* U = arena + off;
        off += (size_t)k * 3 * bb[w].nr;
        float* V = arena + off;
        off += (size_t)k * 3 * bb[w].nc;
        h->info.rank_sum += k;
        h->info.rank_max = std::max(h->info.rank_max, k);
        h->info.factor_bytes += (long long)sizeof(float) * k * 3 * (bb[w].nr + bb[w].nc);
        if (k > 0) {
            const long long nr3 = 3LL * bb[w].nr, nc3 = 3LL * bb[w].nc;
            dim3 blk(32, 8);
            k_transpose<<<dim3((unsigned)((nr3 + 31) / 32), (k + 31) / 32), blk, 0, st>>>(d_w + bb[w].offU, U, nr3, k);
            k_transpose<<<dim3((unsigned)((nc3 + 31) / 32), (k + 31) / 32), blk, 0, st>>>(d_w + bb[w].offV, V, nc3, k);
            WCHK(cudaGetLastError());
        }
        h->factor_ptrs[bi] = {U, V};
    }
    WCHK(cudaStreamSynchronize(st));
    cleanup();
    return FBC_OK;
#undef WALLOC
#undef WCHK
}

}  // namespace

extern "C" {

int fbc_hmat_partition(const int32_t* xy_i, int32_t n_i, const int32_t* xy_p, int32_t n_p, int32_t L, double c,
                       double gamma, int32_t b_min, int64_t* n_blocks, int64_t* blocks, int64_t cap, int64_t* perm_p,
                       int64_t* perm_i) {
    fbc::report_error(FBC_OK, "");
    if (!n_blocks) return hfail(FBC_ERR_INVALID_ARG, "n_blocks is NULL");
    int rc = check_partition_args(xy_i, n_i, xy_p, n_p, L, c, gamma, b_min);
    if (rc) return rc;
    Tree Tp, Ti;
    build_tree(xy_p, n_p, L, c, b_min, Tp);
    build_tree(xy_i, n_i, L, c, b_min, Ti);
    std::vector<BlockRec> bl;
    partition(Tp, Ti, gamma, (double)L * c, bl);
    *n_blocks = (int64_t)bl.size();
    if (blocks) {
        if (cap < (int64_t)bl.size()) return hfail(FBC_ERR_INVALID_ARG, "blocks: capacity too small");
        for (size_t i = 0; i < bl.size(); i++) {
            const int64_t v[5] = {bl[i].r0, bl[i].nr, bl[i].c0, bl[i].nc, bl[i].lowrank};
            memcpy(blocks + 5 * i, v, sizeof(v));
        }
    }
    if (perm_p) memcpy(perm_p, Tp.perm.data(), sizeof(int64_t) * Tp.perm.size());
    if (perm_i) memcpy(perm_i, Ti.perm.data(), sizeof(int64_t) * Ti.perm.size());
    return FBC_OK;
}

int fbc_hmat_create(fbc_plan* plan, const fbc_hmat_options* opt_in, void* stream, fbc_hmat** out) {
    fbc::report_error(FBC_OK, "");
    if (!out) return hfail(FBC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    fbc_hmat_options opt{1e-5, 2.0, 20, 0, 0};
    if (opt_in) opt = *opt_in;
    if (opt.max_rank == 0) opt.max_rank = kDefaultMaxRank;
    if (!(opt.eps >= 1e-6 && opt.eps < 1.0)) return hfail(FBC_ERR_INVALID_ARG, "eps must be in [1e-6, 1)");
    if (!(opt.gamma > 0.0) || !std::isfinite(opt.gamma)) return hfail(FBC_ERR_INVALID_ARG, "gamma must be positive");
    if (opt.b_min < 1 || opt.b_min > 64) return hfail(FBC_ERR_INVALID_ARG, "b_min must be in 1..64");
    if (opt.max_rank < 1 || opt.max_rank > kMaxRank) return hfail(FBC_ERR_INVALID_ARG, "max_rank must be in 0..6141");
    if (opt.scratch_bytes < 0) return hfail(FBC_ERR_INVALID_ARG, "scratch_bytes must be >= 0");
    if (!plan) return hfail(FBC_ERR_INVALID_ARG, "plan is NULL");
    fbc::Plan& P = plan->p;
    if (P.host_only) return hfail(FBC_ERR_INVALID_ARG, "host-only plan");
    if (P.opt.flags & FBC_PLAN_SELF_TERMS)
        return hfail(FBC_ERR_UNSUPPORTED, "H-matrix: plans with self-terms use the lattice kernel");
    if (P.opt.flags & fbc::kPlanNearFieldSet)
        return hfail(FBC_ERR_UNSUPPORTED, "H-matrix: the plan has a lattice near field");
    std::vector<int32_t> xy_i, xy_p;
    original_sites(P.perm_i, P.xy_i_sorted, P.n_i, xy_i);
    original_sites(P.perm_p, P.xy_p_sorted, P.n_p, xy_p);
    int rc = check_partition_args(xy_i.data(), P.n_i, xy_p.data(), P.n_p, P.L, P.c, opt.gamma, opt.b_min);
    if (rc) return rc;
    const auto t_start = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    fbc_hmat* h = new fbc_hmat();
    h->n_i = P.n_i, h->n_p = P.n_p, h->L = P.L, h->opt = opt;
    Tree Tp, Ti;
    build_tree(xy_p.data(), P.n_p, P.L, P.c, opt.b_min, Tp);
    build_tree(xy_i.data(), P.n_i, P.L, P.c, opt.b_min, Ti);
    partition(Tp, Ti, opt.gamma, (double)P.L * P.c, h->blocks);
    const int nbk = (int)h->blocks.size();
    h->ranks.assign(nbk, 0);
    h->factor_ptrs.assign(nbk, {nullptr, nullptr});
    fbc_hmat_info& I = h->info;
    I.n_rows = 3LL * P.n_p * P.L, I.n_cols = 3LL * P.n_i * P.L;
    for (const auto& b : h->blocks) (b.lowrank ? I.n_lowrank : I.n_dense)++;
    for (int n = 0; n < (int)Tp.start.size(); n++) I.n_row_leaves += Tp.leaf(n);
    for (int n = 0; n < (int)Ti.start.size(); n++) I.n_col_leaves += Ti.leaf(n);
    const long long n_pat = (long long)P.n_p * P.L, n_iat = (long long)P.n_i * P.L;
#define CALLOC(p, n, what)                  \
    do {                                    \
        if ((rc = halloc(&(p), (n), what))) { \
            free_hmat(h);                   \
            return rc;                      \
        }                                   \
    } while (0)
#define CCHK(call)                     \
    do {                               \
        cudaError_t e_ = (call);       \
        if (e_ != cudaSuccess) {       \
            rc = hcuda(e_, #call);     \
            free_hmat(h);              \
            return rc;                 \
        }                              \
    } while (0)
    // cluster-order atoms and permutations
    {
        std::vector<int4> ra(n_pat), ca(n_iat);
        std::vector<int> pp(n_pat), pi(n_iat);
        for (long long k = 0; k < n_pat; k++) {
            const long long id = Tp.perm[k];
            const int a = (int)(id / P.L), p = (int)(id % P.L);
            ra[k] = make_int4(xy_p[2 * a], xy_p[2 * a + 1], p, 0);
            pp[k] = (int)id;
        }
        for (long long k = 0; k < n_iat; k++) {
            const long long id = Ti.perm[k];
            const int b = (int)(id / P.L), q = (int)(id % P.L);
            ca[k] = make_int4(xy_i[2 * b], xy_i[2 * b + 1], q, 0);
            pi[k] = (int)id;
        }
        CALLOC(h->d_perm_p, (size_t)n_pat, "hmat_perm");
        CALLOC(h->d_perm_i, (size_t)n_iat, "hmat_perm");
        int4 *d_ra = nullptr, *d_ca = nullptr;
        float* d_tab = nullptr;
        const size_t tab_n = (size_t)P.Dx * P.Dy * (P.L / 2 + 1) * 6;
        auto free_tmp = [&]() {
            if (d_ra) cudaFree(d_ra);
            if (d_ca) cudaFree(d_ca);
            if (d_tab) cudaFree(d_tab);
        };
#define TALLOC(p, n, what)                    \
    do {                                      \
        if ((rc = halloc(&(p), (n), what))) { \
            free_tmp();                       \
            free_hmat(h);                     \
            return rc;                        \
        }                                     \
    } while (0)
#define TCHK(call)                 \
    do {                           \
        cudaError_t e_ = (call);   \
        if (e_ != cudaSuccess) {   \
            rc = hcuda(e_, #call); \
            free_tmp();            \
            free_hmat(h);          \
            return rc;             \
        }                          \
    } while (0)
        TALLOC(d_ra, (size_t)n_pat, "hmat_atoms");
        TALLOC(d_ca, (size_t)n_iat, "hmat_atoms");
        TALLOC(d_tab, tab_n, "hmat_real_space_table");
        TCHK(cudaMemcpyAsync(h->d_perm_p, pp.data(), sizeof(int) * n_pat, cudaMemcpyHostToDevice, st));
        TCHK(cudaMemcpyAsync(h->d_perm_i, pi.data(), sizeof(int) * n_iat, cudaMemcpyHostToDevice, st));
        TCHK(cudaMemcpyAsync(d_ra, ra.data(), sizeof(int4) * n_pat, cudaMemcpyHostToDevice, st));
        TCHK(cudaMemcpyAsync(d_ca, ca.data(), sizeof(int4) * n_iat, cudaMemcpyHostToDevice, st));
        TCHK(fbc::launch_real_space_table(P, d_tab, st));
        Geom g{d_ra, d_ca, d_tab, P.Dx, P.box_x0, P.box_y0, P.L, P.L / 2};
        // dense blocks
        size_t dense_n = 0;
        for (const auto& b : h->blocks)
            if (!b.lowrank) dense_n += (size_t)9 * b.nr * b.nc;
        if (dense_n) {
            float* arena = nullptr;
            TALLOC(arena, dense_n, "hmat_dense");
            h->arenas.push_back(arena);
            size_t off = 0;
            for (int i = 0; i < nbk; i++) {
                const auto& b = h->blocks[i];
                if (b.lowrank) continue;
                const long long pairs = b.nr * b.nc;
                k_dense_fill<<<(unsigned)((pairs + 255) / 256), 256, 0, st>>>(g, (int)b.r0, (int)b.nr, (int)b.c0,
                                                                           (int)b.nc, arena + off);
                h->factor_ptrs[i] = {arena + off, nullptr};
                off += (size_t)9 * b.nr * b.nc;
            }
            TCHK(cudaGetLastError());
            I.dense_bytes = (long long)(sizeof(float) * dense_n);
        }
        // one limit for every build (the attribute belongs to the kernels, not to this object)
        TCHK(cudaFuncSetAttribute(k_aca_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBuildSmemMax));
        TCHK(cudaFuncSetAttribute(k_aca_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBuildSmemMax));
        // low-rank blocks in waves that share the build scratch
        size_t free_b = 0, total_b = 0;
        TCHK(cudaMemGetInfo(&free_b, &total_b));
        const long long budget = opt.scratch_bytes ? opt.scratch_bytes : (long long)(0.4 * (double)free_b);
        std::vector<int> lr;
        for (int i = 0; i < nbk; i++)
            if (h->blocks[i].lowrank) lr.push_back(i);
        auto cost = [&](int i) {
            const auto& b = h->blocks[i];
            const long long kc = std::min<long long>(std::min(3 * b.nr, 3 * b.nc), opt.max_rank) + 3;
            return (long long)sizeof(float) * kc * 3 * (b.nr + b.nc) * 21 / 20;  // factors + partials
        };
        std::stable_sort(lr.begin(), lr.end(), [&](int a, int b) { return cost(a) > cost(b); });
        size_t pos = 0;
        while (pos < lr.size()) {
            std::vector<int> wave{lr[pos++]};
            long long used = cost(wave[0]);
            while (pos < lr.size() && used + cost(lr[pos]) <= budget) used += cost(lr[pos]), wave.push_back(lr[pos++]);
            I.n_waves++;
            if ((rc = build_wave(h, wave, g, st))) {
                free_tmp();
                free_hmat(h);
                return rc;
            }
        }
        TCHK(cudaStreamSynchronize(st));
        free_tmp();
#undef TALLOC
#undef TCHK
    }
    // apply structures: blocks, z items, leaves and their covering blocks
    std::vector<ApplyBlk> ab(nbk);
    std::vector<int2> zit;
    std::vector<long long> zoff;
    long long zp_total = 0, z_total = 0;
    for (int i = 0; i < nbk; i++) {
        const auto& b = h->blocks[i];
        ApplyBlk& a = ab[i];
        a.U = h->factor_ptrs[i].first, a.V = h->factor_ptrs[i].second;
        a.r0 = (int)b.r0, a.nr = (int)b.nr, a.c0 = (int)b.c0, a.nc = (int)b.nc;
        a.lowrank = (int)b.lowrank, a.k = b.lowrank ? h->ranks[i] : 0;
        a.offZ = z_total, a.zit0 = (int)zit.size(), a.n_zit = 0;
        if (b.lowrank && a.k > 0) {
            z_total += (long long)kRG * a.k;
            for (long long j = 0, c = 0; j < 3 * b.nc; j += kZCols, c++) {
                zit.push_back(make_int2(i, (int)c));
                zoff.push_back(zp_total);
                zp_total += (long long)kRG * a.k;
            }
            a.n_zit = (int)zit.size() - a.zit0;
        }
        h->max_k = std::max(h->max_k, a.k);
    }
    std::vector<int> leaf_r0, leaf_nr;
    for (int n = 0; n < (int)Tp.start.size(); n++)
        if (Tp.leaf(n)) leaf_r0.push_back((int)Tp.start[n]), leaf_nr.push_back((int)Tp.count[n]);
    {  // leaves in cluster order
        std::vector<int> idx(leaf_r0.size());
        std::iota(idx.begin(), idx.end(), 0);
        std::sort(idx.begin(), idx.end(), [&](int a, int b) { return leaf_r0[a] < leaf_r0[b]; });
        std::vector<int> r0s, nrs;
        for (int i : idx) r0s.push_back(leaf_r0[i]), nrs.push_back(leaf_nr[i]);
        leaf_r0.swap(r0s), leaf_nr.swap(nrs);
    }
    h->n_leaves = (int)leaf_r0.size();
    for (int n : leaf_nr) h->max_leaf_rows = std::max(h->max_leaf_rows, 3 * n);
    std::vector<std::vector<int>> cov(h->n_leaves);
    for (int i = 0; i < nbk; i++) {
        const auto& b = h->blocks[i];
        if (b.lowrank && ab[i].k == 0) continue;  // an exactly zero block
        int lf = (int)(std::lower_bound(leaf_r0.begin(), leaf_r0.end(), (int)b.r0) - leaf_r0.begin());
        for (; lf < h->n_leaves && leaf_r0[lf] < b.r0 + b.nr; lf++) cov[lf].push_back(i);
    }
    std::vector<int> cover_off(h->n_leaves + 1, 0), cover;
    for (int lf = 0; lf < h->n_leaves; lf++) {
        cover.insert(cover.end(), cov[lf].begin(), cov[lf].end());
        cover_off[lf + 1] = (int)cover.size();
    }
    CALLOC(h->d_blocks, (size_t)nbk, "hmat_apply");
    CALLOC(h->d_leaf_r0, (size_t)h->n_leaves, "hmat_apply");
    CALLOC(h->d_leaf_nr, (size_t)h->n_leaves, "hmat_apply");
    CALLOC(h->d_cover_off, (size_t)h->n_leaves + 1, "hmat_apply");
    CALLOC(h->d_cover, std::max<size_t>(cover.size(), 1), "hmat_apply");
    h->n_zitems = (int)zit.size();
    CALLOC(h->d_zitems, std::max<size_t>(zit.size(), 1), "hmat_apply");
    CALLOC(h->d_zp_off, std::max<size_t>(zoff.size(), 1), "hmat_apply");
    CALLOC(h->d_x, (size_t)kRG * 3 * n_iat, "hmat_workspace");
    CALLOC(h->d_zp, (size_t)std::max(zp_total, 1LL), "hmat_workspace");
    CALLOC(h->d_z, (size_t)std::max(z_total, 1LL), "hmat_workspace");
    CALLOC(h->d_fpart, (size_t)kRG * kFParts * 3, "hmat_workspace");
    CALLOC(h->d_mean, (size_t)kRG * 3, "hmat_workspace");
    CALLOC(h->d_usum, (size_t)kRG * h->n_leaves * 3, "hmat_workspace");
    CCHK(cudaMemcpyAsync(h->d_blocks, ab.data(), sizeof(ApplyBlk) * nbk, cudaMemcpyHostToDevice, st));
    CCHK(cudaMemcpyAsync(h->d_leaf_r0, leaf_r0.data(), sizeof(int) * h->n_leaves, cudaMemcpyHostToDevice, st));
    CCHK(cudaMemcpyAsync(h->d_leaf_nr, leaf_nr.data(), sizeof(int) * h->n_leaves, cudaMemcpyHostToDevice, st));
    CCHK(cudaMemcpyAsync(h->d_cover_off, cover_off.data(), sizeof(int) * (h->n_leaves + 1), cudaMemcpyHostToDevice, st));
    if (!cover.empty())
        CCHK(cudaMemcpyAsync(h->d_cover, cover.data(), sizeof(int) * cover.size(), cudaMemcpyHostToDevice, st));
    if (!zit.empty()) {
        CCHK(cudaMemcpyAsync(h->d_zitems, zit.data(), sizeof(int2) * zit.size(), cudaMemcpyHostToDevice, st));
        CCHK(cudaMemcpyAsync(h->d_zp_off, zoff.data(), sizeof(long long) * zoff.size(), cudaMemcpyHostToDevice, st));
    }
    h->apply_smem = sizeof(double) * (size_t)h->max_leaf_rows * kRG;  // at most 64 atoms: 6 KB
    CCHK(cudaStreamSynchronize(st));
    cudaGetDevice(&h->device);
    I.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    *out = h;
    return FBC_OK;
#undef CALLOC
#undef CCHK
}

int fbc_hmat_apply(fbc_hmat* h, const double* f, double* u, int32_t n_rhs, double alpha, double beta, uint32_t flags,
                   void* stream) {
    fbc::report_error(FBC_OK, "");
    if (!h || !f || !u) return hfail(FBC_ERR_INVALID_ARG, "NULL argument");
    if (n_rhs < 1) return hfail(FBC_ERR_INVALID_ARG, "n_rhs must be >= 1");
    if (flags & ~(FBC_APPLY_PROJECT_NEUTRAL | FBC_APPLY_ZERO_MEAN_U)) return hfail(FBC_ERR_INVALID_ARG, "unknown flags");
    cudaStream_t st = (cudaStream_t)stream;
    const long long n_iat = (long long)h->n_i * h->L, n_pat = (long long)h->n_p * h->L;
    const bool project = flags & FBC_APPLY_PROJECT_NEUTRAL, zmean = flags & FBC_APPLY_ZERO_MEAN_U;
    cudaError_t e;
#define HLAUNCH(name, ...)                                     \
    do {                                                       \
        __VA_ARGS__;                                           \
        if ((e = cudaGetLastError()) != cudaSuccess) return hcuda(e, "fbc_hmat_apply: " name); \
    } while (0)
    for (int g0 = 0; g0 < n_rhs; g0 += kRG) {
        const int rg = std::min(kRG, n_rhs - g0);
        const double* fg = f + (long long)g0 * n_iat * 3;
        double* ug = u + (long long)g0 * n_pat * 3;
        if (project) {
            HLAUNCH("k_hm_fsum", k_hm_fsum<<<dim3(kFParts, rg), 256, 0, st>>>(fg, n_iat, h->d_fpart));
            HLAUNCH("k_hm_mean", k_hm_mean<<<rg, 32, 0, st>>>(h->d_fpart, kFParts, n_iat, h->d_mean));
        }
        const long long nx = (long long)rg * n_iat * 3;
        HLAUNCH("k_hm_gather", k_hm_gather<<<(unsigned)((nx + 255) / 256), 256, 0, st>>>(
                                   fg, h->d_perm_i, n_iat, rg, project ? h->d_mean : nullptr, h->d_x));
        if (h->n_zitems) {
#define HZ(R) k_hm_z<R><<<h->n_zitems, 256, 0, st>>>(h->d_blocks, h->d_zitems, h->d_x, 3 * n_iat, h->d_zp, h->d_zp_off)
            HLAUNCH("k_hm_z", if (rg == 1) HZ(1); else if (rg == 2) HZ(2); else if (rg == 3) HZ(3); else HZ(4));
#undef HZ
            const unsigned tiles = (unsigned)((rg * h->max_k + 31) / 32);
            HLAUNCH("k_hm_zsum", k_hm_zsum<<<dim3((unsigned)h->blocks.size(), tiles), 256, 0, st>>>(
                                     h->d_blocks, h->d_zp, h->d_zp_off, rg, h->d_z));
        }
#define HY(R)                                                                                                  \
    k_hm_y<R><<<h->n_leaves, 256, h->apply_smem, st>>>(h->d_blocks, h->d_leaf_r0, h->d_leaf_nr, h->d_cover_off,     \
                                                       h->d_cover, h->d_z, h->d_x, 3 * n_iat, h->d_perm_p, n_pat,    \
                                                       alpha, beta, ug, zmean ? h->d_usum : nullptr, h->max_leaf_rows)
        HLAUNCH("k_hm_y", if (rg == 1) HY(1); else if (rg == 2) HY(2); else if (rg == 3) HY(3); else HY(4));
#undef HY
        if (zmean) {
            HLAUNCH("k_hm_mean", k_hm_mean<<<rg, 32, 0, st>>>(h->d_usum, h->n_leaves, n_pat, h->d_mean));
            HLAUNCH("k_hm_usub", k_hm_usub<<<dim3(kFParts, rg), 256, 0, st>>>(ug, n_pat, h->d_mean));
        }
    }
#undef HLAUNCH
    return FBC_OK;
}

int fbc_hmat_get_info(const fbc_hmat* h, fbc_hmat_info* info) {
    fbc::report_error(FBC_OK, "");
    if (!h || !info) return hfail(FBC_ERR_INVALID_ARG, "NULL argument");
    *info = h->info;
    return FBC_OK;
}

int fbc_hmat_blocks(const fbc_hmat* h, int64_t* blocks, int32_t* ranks, int64_t cap) {
    fbc::report_error(FBC_OK, "");
    if (!h) return hfail(FBC_ERR_INVALID_ARG, "NULL argument");
    if ((blocks || ranks) && cap < (int64_t)h->blocks.size())
        return hfail(FBC_ERR_INVALID_ARG, "capacity too small");
    for (size_t i = 0; i < h->blocks.size(); i++) {
        const auto& b = h->blocks[i];
        if (blocks) {
            const int64_t v[5] = {b.r0, b.nr, b.c0, b.nc, b.lowrank};
            memcpy(blocks + 5 * i, v, sizeof(v));
        }
        if (ranks) ranks[i] = b.lowrank ? h->ranks[i] : 0;
    }
    return FBC_OK;
}

void fbc_hmat_destroy(fbc_hmat* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    free_hmat(h);
}

}  // extern "C"
