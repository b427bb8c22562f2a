// Host side of the FBC pad-update library: argument validation, the
// spatially compact tiling of the column sets, the difference-table box,
// device memory ownership and the C ABI entry points declared in fbc.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>

#include "fbc_internal.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? FBC_ERR_OOM : FBC_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define FBC_CUDA(call)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// Recursive bisection along the longer side of the bounding box.  The left
// part always holds a multiple of T sites, so every tile is full except the
// last one.  Ties are broken by the other coordinate and then the index, so
// the order is deterministic on every host.
void bisect(const int32_t* xy, std::vector<int>& idx, int lo, int hi, int T) {
    int n = hi - lo;
    if (n <= T) return;
    int minx = INT32_MAX, maxx = INT32_MIN, miny = INT32_MAX, maxy = INT32_MIN;
    for (int t = lo; t < hi; t++) {
        int x = xy[2 * idx[t]], y = xy[2 * idx[t] + 1];
        minx = std::min(minx, x), maxx = std::max(maxx, x);
        miny = std::min(miny, y), maxy = std::max(maxy, y);
    }
    int ax = (maxx - minx >= maxy - miny) ? 0 : 1;
    std::sort(idx.begin() + lo, idx.begin() + hi, [&](int a, int b) {
        int pa = xy[2 * a + ax], pb = xy[2 * b + ax];
        if (pa != pb) return pa < pb;
        int qa = xy[2 * a + 1 - ax], qb = xy[2 * b + 1 - ax];
        if (qa != qb) return qa < qb;
        return a < b;
    });
    int n_left = T * ((n + 2 * T - 1) / (2 * T));
    if (n_left >= n) n_left = T * ((n - 1) / T);
    bisect(xy, idx, lo, lo + n_left, T);
    bisect(xy, idx, lo + n_left, hi, T);
}

struct Tiling {
    std::vector<int> perm;      // slot -> original index or -1
    std::vector<int2> xy;       // slot -> site (padding: first site of the tile)
    std::vector<int4> bbox;     // tile -> (minx, maxx, miny, maxy)
    int n_tiles = 0, n_pad = 0, max_w = 0, max_h = 0;
};

// row_major: inside each tile, order the sites by (y, x), so that the threads
// of a warp (consecutive rows of a pad tile) gather table cells that are
// neighbours along x -- consecutive shared-memory records, not records a
// sub-box width apart, which share banks.  Each pad column's sum over the
// interface columns keeps its order, so results do not change.
Tiling make_tiling(const int32_t* xy, int n, int T, bool row_major) {
    Tiling t;
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    bisect(xy, idx, 0, n, T);
    if (row_major)
        for (int lo = 0; lo < n; lo += T)
            std::sort(idx.begin() + lo, idx.begin() + std::min(n, lo + T), [&](int a, int b) {
                if (xy[2 * a + 1] != xy[2 * b + 1]) return xy[2 * a + 1] < xy[2 * b + 1];
                if (xy[2 * a] != xy[2 * b]) return xy[2 * a] < xy[2 * b];
                return a < b;
            });
    t.n_tiles = (n + T - 1) / T;
    t.n_pad = t.n_tiles * T;
    t.perm.assign(t.n_pad, -1);
    t.xy.resize(t.n_pad);
    t.bbox.resize(t.n_tiles);
    for (int tile = 0; tile < t.n_tiles; tile++) {
        int4 bb = make_int4(INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN);
        int first = idx[tile * T];
        for (int s = 0; s < T; s++) {
            int slot = tile * T + s;
            int o = (slot < n) ? idx[slot] : -1;
            t.perm[slot] = o;
            int src = (o >= 0) ? o : first;
            int x = xy[2 * src], y = xy[2 * src + 1];
            t.xy[slot] = make_int2(x, y);
            bb.x = std::min(bb.x, x), bb.y = std::max(bb.y, x);
            bb.z = std::min(bb.z, y), bb.w = std::max(bb.w, y);
        }
        t.bbox[tile] = bb;
        t.max_w = std::max(t.max_w, bb.y - bb.x + 1);
        t.max_h = std::max(t.max_h, bb.w - bb.z + 1);
    }
    return t;
}

// Cumulative Richardson weights: with w_i = (n+i)^N (-1)^(i+N) / (i! (N-i)!)
// (Eq. 36), Q0 = sum_i w_i G_{n+i} = G_n + sum_{m=n+1}^{n+N} W_m t_m where
// t_m is the m-th paired image increment and W_m = sum_{i >= m-n} w_i.  The
// increments are small, so this arrangement keeps the rounding of G_n out of
// the large alternating weights.
void richardson_cumulative(int n, int N, double* W) {
    std::vector<double> w(N + 1);
    for (int i = 0; i <= N; i++) {
        double num = 1.0;
        for (int e = 0; e < N; e++) num *= (double)(n + i);
        double den = 1.0;
        for (int t = 2; t <= i; t++) den *= t;
        for (int t = 2; t <= N - i; t++) den *= t;
        w[i] = (((i + N) & 1) ? -num : num) / den;
    }
    for (int m = n + 1; m <= n + N; m++) {
        double s = 0.0;
        for (int i = N; i >= m - n; i--) s += w[i];
        W[m - n - 1] = s;
    }
}

// Full stiffness C_ijkl of the medium in the computational frame and its
// Christoffel form K[I][J] with M_ik = sum_J K[I][J] z_j z_l over the
// symmetric index pairs I = (i, k), J = (j, l).
void christoffel_form(const fbc_material& m, const double Q[9], double K[36]) {
    static const int pr[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
    double C[3][3][3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) {
                    double v = 0.0;
                    if (i == j && k == l) v += m.C12;
                    if (i == k && j == l) v += m.C44;
                    if (i == l && j == k) v += m.C44;
                    if (i == j && j == k && k == l) v += m.C11 - m.C12 - 2.0 * m.C44;
                    C[i][j][k][l] = v;
                }
    double R[3][3][3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) {
                    double v = 0.0;
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            for (int c = 0; c < 3; c++)
                                for (int d = 0; d < 3; d++)
                                    v += Q[3 * a + i] * Q[3 * b + j] * Q[3 * c + k] * Q[3 * d + l] * C[a][b][c][d];
                    R[i][j][k][l] = v;
                }
    for (int I = 0; I < 6; I++)
        for (int J = 0; J < 6; J++) {
            int i = pr[I][0], k = pr[I][1], j = pr[J][0], l = pr[J][1];
            K[6 * I + J] = (j == l) ? R[i][j][k][l] : R[i][j][k][l] + R[i][l][k][j];
        }
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

template <class T>
int dev_alloc(T** p, size_t count, size_t& acc, const char* what) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    if (getenv("FBC_TEST_FAIL_ALLOC") && strcmp(getenv("FBC_TEST_FAIL_ALLOC"), what) == 0)
        return fail(FBC_ERR_OOM, "injected allocation failure: %s", what);
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, what);
    }
    acc += align_up(bytes);
    return FBC_OK;
}

void free_plan(fbc::Plan& P) {
    void* bufs[] = {P.d_xy_p,  P.d_off_i,    P.d_bbox_a, P.d_bbox_b, P.d_perm_i, P.d_perm_p,
                    P.d_used,  P.d_tw,       P.d_twL,    P.d_twl,    P.d_table,  P.d_table32, P.d_table_x2, P.d_table_x2_k0,
                    P.d_fh,    P.d_uh,       P.d_part,   P.d_stage_f, P.d_stage_u, P.d_status, P.d_bprep,
                    P.d_relax, P.d_uh32};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (auto& e : P.ev)
        if (e) cudaEventDestroy(e), e = nullptr;
    for (auto& e : P.host_ev)
        if (e) cudaEventDestroy(e), e = nullptr;
    for (auto& h : P.host_st)
        if (h) cudaStreamDestroy(h), h = nullptr;
    fbc::release_surrogate_buffers(P);
    fbc::fft_free(P);
}

// Allocate the derived table a reduced-precision contraction reads (once).
int ensure_derived(fbc::Plan& P, int precision) {
    const size_t cells = (size_t)P.K * P.Dy * P.Dx;
    size_t acc = 0;
    if ((precision == FBC_PREC_FP32 || fbc::is_tensor_precision(precision)) && !P.d_table32) {
        int s = dev_alloc(&P.d_table32, cells * 6, acc, "table32");
        if (s) return s;
    }
    // the tensor forms' split force operand, sized for this precision's pieces
    if (fbc::is_tensor_precision(precision) && P.bprep_prec != precision) {
        const size_t want = fbc::contract_tc_prep_bytes(P, precision);
        if (P.d_bprep && P.bprep_bytes < want) {
            cudaFree(P.d_bprep);
            P.workspace_bytes -= P.bprep_bytes;
            P.d_bprep = nullptr, P.bprep_bytes = 0;
        }
        if (!P.d_bprep) {
            unsigned char* q = nullptr;
            int s = dev_alloc(&q, want, acc, "tensor force operand");
            if (s) return s;
            P.d_bprep = q, P.bprep_bytes = want;
        }
        P.bprep_prec = precision;
    }
    // the tensor-core forms' modes k >= 1: their group partials are FP32 sums, kept in FP32
    if (fbc::is_tensor_precision(precision) && !P.d_uh32) {
        int s = dev_alloc(&P.d_uh32, (size_t)P.opt.max_rhs * P.K * P.NPpad * 6, acc, "uh32");
        if (s) return s;
    }
    // FBC_PREC_BF16X6: the double-float table and the sliced force operand with its scales
    if (precision == FBC_PREC_BF16X6 && P.bprep_prec != precision) {
        const size_t want = fbc::contract_oz_prep_bytes(P);
        if (P.d_bprep && P.bprep_bytes < want) {
            cudaFree(P.d_bprep);
            P.workspace_bytes -= P.bprep_bytes;
            P.d_bprep = nullptr, P.bprep_bytes = 0;
        }
        if (!P.d_bprep) {
            unsigned char* q = nullptr;
            int s = dev_alloc(&q, want, acc, "sliced force operand");
            if (s) return s;
            P.d_bprep = q, P.bprep_bytes = want;
        }
        P.bprep_prec = precision;
    }
    if ((precision == FBC_PREC_F32X2 || precision == FBC_PREC_BF16X6) && !P.d_table_x2) {
        int s = dev_alloc(&P.d_table_x2, cells * 12, acc, "table_x2");
        if (s) return s;
    }
    // the k = 0 mode of the FP32 and tensor-core forms runs in double-float
    if ((precision == FBC_PREC_FP32 || fbc::is_tensor_precision(precision)) && !P.d_table_x2_k0) {
        int s = dev_alloc(&P.d_table_x2_k0, (size_t)P.Dy * P.Dx * 12, acc, "table_x2_k0");
        if (s) return s;
    }
    P.workspace_bytes += acc;
    return FBC_OK;
}

int validate_material(const fbc_material& m, double Q[9]) {
    bool allzero = true;
    for (int t = 0; t < 9; t++) allzero = allzero && m.Q[t] == 0.0;
    for (int t = 0; t < 9; t++) Q[t] = allzero ? ((t % 4 == 0) ? 1.0 : 0.0) : m.Q[t];
    for (int t = 0; t < 9; t++)
        if (!std::isfinite(Q[t])) return fail(FBC_ERR_INVALID_ARG, "material Q has a non-finite entry");
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += Q[3 * k + i] * Q[3 * k + j];
            if (std::fabs(s - (i == j ? 1.0 : 0.0)) > 1e-12)
                return fail(FBC_ERR_INVALID_ARG, "material Q is not orthogonal");
        }
    if (m.kind == FBC_MATERIAL_ISOTROPIC) {
        if (!(m.mu > 0.0) || !(m.nu > -1.0) || !(m.nu < 0.5) || !std::isfinite(m.mu))
            return fail(FBC_ERR_INVALID_ARG, "isotropic medium needs mu > 0 and -1 < nu < 0.5");
        return FBC_OK;
    }
    if (m.kind == FBC_MATERIAL_CUBIC) {
        if (!(m.C44 > 0.0) || !(m.C11 - m.C12 > 0.0) || !(m.C11 + 2.0 * m.C12 > 0.0) || !std::isfinite(m.C11))
            return fail(FBC_ERR_INVALID_ARG, "cubic medium is not stable (C44 > 0, C11 > |C12|, C11 + 2 C12 > 0)");
        // the line direction must map onto a cube axis (mirror x3 -> -x3 preserved)
        bool ok = false;
        for (int j = 0; j < 3; j++) ok = ok || std::fabs(std::fabs(Q[3 * j + 2]) - 1.0) < 1e-12;
        if (!ok)
            return fail(FBC_ERR_UNSUPPORTED,
                        "cubic medium: the line direction must lie along a cube axis (mirror symmetry)");
        return FBC_OK;
    }
    return fail(FBC_ERR_INVALID_ARG, "unknown material kind %d", m.kind);
}

}  // namespace

int fbc::report_error(int code, const char* msg) {
    g_last_error = msg ? msg : "";
    return code;
}

extern "C" {

const char* fbc_last_error(void) { return g_last_error.c_str(); }

const char* fbc_version(void) { return "fbc-gb300 0.1 (sm_103a)"; }

void fbc_default_options(fbc_options* opt) {
    if (!opt) return;
    opt->precision = FBC_PREC_FP64;
    opt->rich_n = 4;
    opt->rich_N = 6;
    opt->quad = 64;
    opt->max_rhs = 1;
    opt->flags = 0;
}

int fbc_plan_create(const fbc_geometry* geom, const fbc_material* mat, const fbc_options* opt_in,
                    fbc_plan** out) {
    g_last_error.clear();
    if (!out) return fail(FBC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!geom || !mat) return fail(FBC_ERR_INVALID_ARG, "geometry or material is NULL");
    fbc_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        fbc_default_options(&opt);
    const int n_i = geom->n_i, n_p = geom->n_p, L = geom->L;
    if (n_i < 1 || n_p < 1) return fail(FBC_ERR_INVALID_ARG, "n_i and n_p must be >= 1");
    if (n_i > (1 << 24) || n_p > (1 << 24)) return fail(FBC_ERR_INVALID_ARG, "too many columns");
    if (!is_pow2(L) || L < 2 || L > 4096) return fail(FBC_ERR_INVALID_ARG, "L must be a power of two in [2, 4096]");
    if (!(geom->c > 0.0) || !std::isfinite(geom->c)) return fail(FBC_ERR_INVALID_ARG, "c must be positive");
    if (!geom->xy_i || !geom->xy_p) return fail(FBC_ERR_INVALID_ARG, "site lists are NULL");
    if (opt.rich_n < 1 || opt.rich_N < 0 || opt.rich_n + opt.rich_N > fbc::kMaxRichImages || opt.rich_N > 12)
        return fail(FBC_ERR_INVALID_ARG, "Richardson needs n >= 1, 0 <= N <= 12, n + N <= %d", fbc::kMaxRichImages);
    if (opt.quad < 8 || opt.quad > fbc::kMaxQuad) return fail(FBC_ERR_INVALID_ARG, "quad must be in [8, %d]", fbc::kMaxQuad);
    if (opt.max_rhs < 1 || opt.max_rhs > 4096) return fail(FBC_ERR_INVALID_ARG, "max_rhs must be in [1, 4096]");
    if (opt.precision < FBC_PREC_FP64 || opt.precision > FBC_PREC_BF16X6)
        return fail(FBC_ERR_INVALID_ARG, "unknown precision %d", opt.precision);
    if (opt.flags & ~(FBC_PLAN_HOST_ONLY | FBC_PLAN_TC_FAST_ACCUMULATE | FBC_PLAN_SELF_TERMS))
        return fail(FBC_ERR_INVALID_ARG, "unknown options.flags bits 0x%x", opt.flags);
    const int32_t coord_lim = 1 << 20;
    for (int t = 0; t < 2 * n_i; t++)
        if (geom->xy_i[t] < -coord_lim || geom->xy_i[t] > coord_lim)
            return fail(FBC_ERR_INVALID_ARG, "interface site coordinate out of range");
    for (int t = 0; t < 2 * n_p; t++)
        if (geom->xy_p[t] < -coord_lim || geom->xy_p[t] > coord_lim)
            return fail(FBC_ERR_INVALID_ARG, "pad site coordinate out of range");
    double Q[9];
    int st = validate_material(*mat, Q);
    if (st) return st;

    // duplicates within each set
    auto has_dup = [](const int32_t* xy, int n) {
        std::vector<int64_t> keys(n);
        for (int t = 0; t < n; t++) keys[t] = ((int64_t)xy[2 * t] << 32) ^ (uint32_t)xy[2 * t + 1];
        std::sort(keys.begin(), keys.end());
        return std::adjacent_find(keys.begin(), keys.end()) != keys.end();
    };
    if (has_dup(geom->xy_i, n_i)) return fail(FBC_ERR_INVALID_ARG, "duplicate interface site");
    if (has_dup(geom->xy_p, n_p)) return fail(FBC_ERR_INVALID_ARG, "duplicate pad site");

    fbc_plan* plan = new (std::nothrow) fbc_plan();
    if (!plan) return fail(FBC_ERR_OOM, "host allocation of the plan failed");
    fbc::Plan& P = plan->p;
    P.host_only = (opt.flags & FBC_PLAN_HOST_ONLY) != 0;
    if (!P.host_only) cudaGetDevice(&P.device);
    P.n_i = n_i, P.n_p = n_p, P.L = L, P.K = L / 2 + 1, P.c = geom->c;
    P.logL = 0;
    while ((1 << P.logL) < L) P.logL++;
    P.opt = opt;
    P.precision = opt.precision;

    // tiling
    fbc::Plan* pp = &P;
    Tiling ta = make_tiling(geom->xy_p, n_p, P.TA, true);
    Tiling tb = make_tiling(geom->xy_i, n_i, P.TB, false);
    P.n_ta = ta.n_tiles, P.n_tb = tb.n_tiles, P.NPpad = ta.n_pad, P.NIpad = tb.n_pad;
    P.W = ta.max_w + tb.max_w - 1;
    P.H = ta.max_h + tb.max_h - 1;
    P.perm_p = ta.perm;
    P.perm_i = tb.perm;
    P.xy_p_sorted = ta.xy;
    P.xy_i_sorted = tb.xy;

    // difference box and the differences that occur
    int pminx = INT32_MAX, pmaxx = INT32_MIN, pminy = INT32_MAX, pmaxy = INT32_MIN;
    int iminx = INT32_MAX, imaxx = INT32_MIN, iminy = INT32_MAX, imaxy = INT32_MIN;
    for (int t = 0; t < n_p; t++) {
        pminx = std::min(pminx, geom->xy_p[2 * t]), pmaxx = std::max(pmaxx, geom->xy_p[2 * t]);
        pminy = std::min(pminy, geom->xy_p[2 * t + 1]), pmaxy = std::max(pmaxy, geom->xy_p[2 * t + 1]);
    }
    for (int t = 0; t < n_i; t++) {
        iminx = std::min(iminx, geom->xy_i[2 * t]), imaxx = std::max(imaxx, geom->xy_i[2 * t]);
        iminy = std::min(iminy, geom->xy_i[2 * t + 1]), imaxy = std::max(imaxy, geom->xy_i[2 * t + 1]);
    }
    P.box_x0 = pminx - imaxx;
    P.box_y0 = pminy - imaxy;
    P.Dx = (pmaxx - iminx) - P.box_x0 + 1;
    P.Dy = (pmaxy - iminy) - P.box_y0 + 1;
    if ((double)P.Dx * P.Dy > 64.0 * 1024 * 1024) {
        delete plan;
        return fail(FBC_ERR_INVALID_ARG, "difference box %d x %d is too large", pp->Dx, pp->Dy);
    }
    std::vector<uint8_t> used((size_t)P.Dx * P.Dy, 0);
    for (int a = 0; a < n_p; a++) {
        int xa = geom->xy_p[2 * a] - P.box_x0, ya = geom->xy_p[2 * a + 1] - P.box_y0;
        for (int b = 0; b < n_i; b++) {
            int ix = xa - geom->xy_i[2 * b], iy = ya - geom->xy_i[2 * b + 1];
            used[(size_t)iy * P.Dx + ix] = 1;
        }
    }
    int zx = -P.box_x0, zy = -P.box_y0;
    if (!(opt.flags & FBC_PLAN_SELF_TERMS) && zx >= 0 && zx < P.Dx && zy >= 0 && zy < P.Dy &&
        used[(size_t)zy * P.Dx + zx]) {
        delete plan;
        return fail(FBC_ERR_INVALID_ARG, "an interface site coincides with a pad site (d = 0 is singular)");
    }
    std::vector<int2> used_list;
    for (int iy = 0; iy < P.Dy; iy++)
        for (int ix = 0; ix < P.Dx; ix++)
            if (used[(size_t)iy * P.Dx + ix]) used_list.push_back(make_int2(ix + P.box_x0, iy + P.box_y0));
    P.n_used = (int)used_list.size();

    // material for the device
    P.mat.kind = mat->kind;
    P.mat.nquad = opt.quad;
    if (mat->kind == FBC_MATERIAL_ISOTROPIC) {
        P.mat.kelvin_pre = 1.0 / (16.0 * M_PI * mat->mu * (1.0 - mat->nu));
        P.mat.kelvin_a = 3.0 - 4.0 * mat->nu;
    } else {
        christoffel_form(*mat, Q, P.mat.K);
    }
    P.tp.L = L, P.tp.K = P.K, P.tp.Lh = L / 2, P.tp.c = P.c;
    P.tp.rich_n = opt.rich_n, P.tp.rich_N = opt.rich_N;
    richardson_cumulative(opt.rich_n, opt.rich_N, P.tp.W);
    P.tp.box_x0 = P.box_x0, P.tp.box_y0 = P.box_y0, P.tp.Dx = P.Dx, P.tp.Dy = P.Dy;

    if (P.host_only) {
        *out = plan;
        return FBC_OK;
    }

    // device buffers
    size_t acc = 0;
    std::vector<int> off_i(P.NIpad);
    for (int s = 0; s < P.NIpad; s++) off_i[s] = tb.xy[s].x + P.W * tb.xy[s].y;
    const size_t cells = (size_t)P.K * P.Dy * P.Dx;
    const int nlb = P.NPpad / fbc::line_cols(L);
#define ALLOC(ptr, n, what)                                  \
    do {                                                     \
        int s_ = dev_alloc(&(ptr), (n), acc, what);          \
        if (s_) {                                            \
            free_plan(P);                                    \
            delete plan;                                     \
            return s_;                                       \
        }                                                    \
    } while (0)
    ALLOC(P.d_xy_p, P.NPpad, "xy_p");
    ALLOC(P.d_off_i, P.NIpad, "off_i");
    ALLOC(P.d_bbox_a, P.n_ta, "bbox_a");
    ALLOC(P.d_bbox_b, P.n_tb, "bbox_b");
    ALLOC(P.d_perm_i, P.NIpad, "perm_i");
    ALLOC(P.d_perm_p, P.NPpad, "perm_p");
    ALLOC(P.d_used, P.n_used, "used");
    ALLOC(P.d_tw, L / 2 + L / 4 + 1, "twiddles");  // L/2 double2, then L/2 float2
    ALLOC(P.d_twL, L, "table_twiddles");
    ALLOC(P.d_twl, L, "line_twiddles");
    size_t ws_before_table = acc;
    ALLOC(P.d_table, cells * 6, "table");
    P.table_bytes = acc - ws_before_table;
    ALLOC(P.d_fh, (size_t)opt.max_rhs * P.K * P.NIpad * 6, "fh");
    ALLOC(P.d_uh, (size_t)opt.max_rhs * P.K * P.NPpad * 6, "uh");
    ALLOC(P.d_part, (size_t)opt.max_rhs * nlb * 3, "partials");
    ALLOC(P.d_relax, (size_t)opt.max_rhs * (fbc::kRelaxBlocks * 2 + nlb), "relaxation");
    ALLOC(P.d_status, 1, "status");
#undef ALLOC
    P.workspace_bytes = acc - P.table_bytes;
    if (int s_ = ensure_derived(P, P.precision)) {
        free_plan(P);
        delete plan;
        return s_;
    }

    std::vector<double2> tw(L / 2 + L / 4 + 1), twL(L);
    std::vector<float2> twl(L);
    P.line_fft = fbc::fft::make_fft(L);
    float2* tw32 = (float2*)(tw.data() + L / 2);  // the FP32 transforms' copy, rounded from FP64
    for (int t = 0; t < L / 2; t++) {
        double ang = 2.0 * M_PI * (double)t / (double)L;
        tw[t] = make_double2(cos(ang), -sin(ang));
        tw32[t] = make_float2((float)tw[t].x, (float)tw[t].y);
    }
    for (int t = 0; t < L; t++) {
        double ang = 2.0 * M_PI * (double)t / (double)L;
        twL[t] = make_double2(cos(ang), sin(ang));
        twl[t] = make_float2((float)cos(ang), (float)-sin(ang));
    }
    cudaError_t e = cudaSuccess;
#define UP(dst, src, n)                                                                   \
    if (e == cudaSuccess) e = cudaMemcpy((dst), (src), sizeof(*(dst)) * (size_t)(n), cudaMemcpyHostToDevice)
    UP(P.d_xy_p, ta.xy.data(), P.NPpad);
    UP(P.d_off_i, off_i.data(), P.NIpad);
    UP(P.d_bbox_a, ta.bbox.data(), P.n_ta);
    UP(P.d_bbox_b, tb.bbox.data(), P.n_tb);
    UP(P.d_perm_i, tb.perm.data(), P.NIpad);
    UP(P.d_perm_p, ta.perm.data(), P.NPpad);
    if (P.n_used) UP(P.d_used, used_list.data(), P.n_used);
    UP(P.d_tw, tw.data(), L / 2 + L / 4 + 1);
    UP(P.d_twL, twL.data(), L);
    UP(P.d_twl, twl.data(), L);
#undef UP
    if (e == cudaSuccess) e = cudaMemset(P.d_table, 0, cells * 6 * sizeof(double));
    // padding columns of fh stay zero for ever: the forward transform never writes them
    if (e == cudaSuccess) e = cudaMemset(P.d_fh, 0, (size_t)opt.max_rhs * P.K * P.NIpad * 6 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(P.d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        int s = cuda_fail(e, "plan upload");
        free_plan(P);
        delete plan;
        return s;
    }
    *out = plan;
    return FBC_OK;
}

int fbc_tabulate_kernel(fbc_plan* plan, void* stream) {
    g_last_error.clear();
    if (!plan) return fail(FBC_ERR_INVALID_ARG, "plan is NULL");
    fbc::Plan& P = plan->p;
    if (P.host_only) return fail(FBC_ERR_INVALID_ARG, "host-only plan");
    if (P.tables_released) return fail(FBC_ERR_UNSUPPORTED, "the plan's tables were released for its surrogate");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = fbc::launch_tabulate(P, st);
    if (e != cudaSuccess) return cuda_fail(e, "tabulate");
    P.tabulated = true;
    P.opt.flags &= ~fbc::kPlanNearFieldSet;  // a new continuum table: the near field must be set again
    if (fbc::is_fft_precision(P.precision)) {
        if (int s = fbc::fft_prepare(P, P.precision)) return s;
    }
    if (P.precision != FBC_PREC_FP64) {
        e = fbc::launch_derive_tables(P, P.precision, st);
        if (e != cudaSuccess) return cuda_fail(e, "derive tables");
    }
    return FBC_OK;
}

int fbc_plan_set_precision(fbc_plan* plan, int32_t precision) {
    g_last_error.clear();
    if (!plan) return fail(FBC_ERR_INVALID_ARG, "plan is NULL");
    if (precision < FBC_PREC_FP64 || precision > FBC_PREC_BF16X6)
        return fail(FBC_ERR_INVALID_ARG, "unknown precision %d", precision);
    fbc::Plan& P = plan->p;
    if (P.host_only) return fail(FBC_ERR_INVALID_ARG, "host-only plan");
    if (P.tables_released) return fail(FBC_ERR_UNSUPPORTED, "the plan's tables were released for its surrogate");
    if (P.sur && precision != FBC_PREC_FP32 && !fbc::is_tensor_precision(precision))
        return fail(FBC_ERR_UNSUPPORTED, "detach the surrogate before switching to this precision");
    if (int st = ensure_derived(P, precision)) return st;
    if (fbc::is_fft_precision(precision) && P.tabulated) {
        if (int st = fbc::fft_prepare(P, precision)) return st;
    }
    P.precision = precision;
    if (P.tabulated && precision != FBC_PREC_FP64) {
        cudaError_t e = fbc::launch_derive_tables(P, precision, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "derive tables");
    }
    return FBC_OK;
}

// Checks shared by the apply entry points.
static int apply_checks(fbc::Plan& P, const double* f, const double* u, int32_t n_rhs, uint32_t flags) {
    if (P.host_only) return fail(FBC_ERR_INVALID_ARG, "host-only plan");
    if (!P.tabulated) return fail(FBC_ERR_NOT_TABULATED, "fbc_apply before fbc_tabulate_kernel");
    if ((P.opt.flags & FBC_PLAN_SELF_TERMS) && !(P.opt.flags & fbc::kPlanNearFieldSet))
        return fail(FBC_ERR_INVALID_ARG, "a plan with self-terms needs the lattice near field before an apply");
    if (P.tables_released && !P.sur) return fail(FBC_ERR_INVALID_ARG, "tables released without a surrogate");
    if (!f || !u) return fail(FBC_ERR_INVALID_ARG, "f or u is NULL");
    if (n_rhs < 1 || n_rhs > P.opt.max_rhs)
        return fail(FBC_ERR_INVALID_ARG, "n_rhs = %d outside [1, max_rhs = %d]", n_rhs, P.opt.max_rhs);
    if (flags & ~(FBC_APPLY_PROJECT_NEUTRAL | FBC_APPLY_ZERO_MEAN_U))
        return fail(FBC_ERR_INVALID_ARG, "unknown apply flags 0x%x", flags);
    const size_t fb = (size_t)n_rhs * P.n_i * P.L * 3 * sizeof(double);
    const size_t ub = (size_t)n_rhs * P.n_p * P.L * 3 * sizeof(double);
    const char* fc = (const char*)f;
    const char* uc = (const char*)u;
    if (fc < uc + ub && uc < fc + fb) return fail(FBC_ERR_INVALID_ARG, "f and u overlap");
    if ((P.precision == FBC_PREC_FP32 || fbc::is_tensor_precision(P.precision)) && !P.d_table32 && !P.sur)
        return fail(FBC_ERR_INVALID_ARG, "FP32 table missing");
    if (fbc::is_tensor_precision(P.precision) && fbc::contract_tc_smem(P.precision, P.W * P.H) > 227 * 1024)
        return fail(FBC_ERR_UNSUPPORTED, "tensor-core contraction: staged sub-box too large for shared memory");
    if ((P.precision == FBC_PREC_F32X2 || P.precision == FBC_PREC_BF16X6) && !P.d_table_x2)
        return fail(FBC_ERR_INVALID_ARG, "double-float table missing");
    if (P.precision == FBC_PREC_BF16X6 && fbc::contract_oz_smem(P.W * P.H) > 227 * 1024)
        return fail(FBC_ERR_UNSUPPORTED, "BF16X6 contraction: staged sub-box too large for shared memory");
    if (fbc::is_fft_precision(P.precision) && !fbc::fft_ready(P, P.precision))
        return fail(FBC_ERR_INVALID_ARG, "in-plane FFT grid missing");
    return FBC_OK;
}

// Forward transform and per-mode contraction: leaves the contracted modes in P.d_uh.
static int apply_modes(fbc::Plan& P, const double* f, int32_t n_rhs, uint32_t flags, cudaStream_t st) {
    if (P.timing) FBC_CUDA(cudaEventRecord(P.ev[0], st));
    cudaError_t e = fbc::launch_forward(P, f, n_rhs, (flags & FBC_APPLY_PROJECT_NEUTRAL) != 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "forward transform");
    if (P.timing) FBC_CUDA(cudaEventRecord(P.ev[1], st));
    if (P.sur) {
        // k = 0 exact (double-float slice), modes k >= 1 from streamed slices
        fbc::ContractArgs A0 = fbc::make_contract_args(P);
        e = fbc::launch_contract_x2_k0(P, A0, n_rhs, st);
        if (e == cudaSuccess) e = fbc::launch_contract_streamed(P, n_rhs, st);
    } else {
        e = fbc::launch_contract(P, n_rhs, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "mode contraction");
    if (P.timing) FBC_CUDA(cudaEventRecord(P.ev[2], st));
    return FBC_OK;
}

static int apply_common(fbc::Plan& P, const double* f, double* u, int32_t n_rhs, double alpha, double beta,
                        uint32_t flags, cudaStream_t st) {
    if (int s = apply_checks(P, f, u, n_rhs, flags)) return s;
    if (!std::isfinite(alpha) || !std::isfinite(beta)) return fail(FBC_ERR_INVALID_ARG, "alpha/beta not finite");
    if (int s = apply_modes(P, f, n_rhs, flags, st)) return s;
    cudaError_t e = fbc::launch_inverse(P, u, n_rhs, alpha, beta, (flags & FBC_APPLY_ZERO_MEAN_U) != 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "inverse transform");
    if (P.timing) {
        FBC_CUDA(cudaEventRecord(P.ev[3], st));
        P.timed_once = true;
    }
    return FBC_OK;
}

int fbc_apply(fbc_plan* plan, const double* f, double* u, int32_t n_rhs, double alpha, double beta,
              uint32_t flags, void* stream) {
    g_last_error.clear();
    if (!plan) return fail(FBC_ERR_INVALID_ARG, "plan is NULL");
    return apply_common(plan->p, f, u, n_rhs, alpha, beta, flags, (cudaStream_t)stream);
}

int fbc_apply_relaxed(fbc_plan* plan, const double* f_new, const double* f_old, double* u, int32_t n_rhs,
                      double* alpha_io, double du_max, uint32_t flags, void* stream) {
    g_last_error.clear();
    if (!plan) return fail(FBC_ERR_INVALID_ARG, "plan is NULL");
    fbc::Plan& P = plan->p;
    if (int s = apply_checks(P, f_new, u, n_rhs, flags)) return s;
    if (!alpha_io) return fail(FBC_ERR_INVALID_ARG, "alpha_io is NULL");
    if (!std::isfinite(du_max) || du_max < 0.0) return fail(FBC_ERR_INVALID_ARG, "du_max must be finite and >= 0");
    if (f_old) {
        if (f_old == f_new) return fail(FBC_ERR_INVALID_ARG, "f_old and f_new are the same buffer");
        if (int s = apply_checks(P, f_old, u, n_rhs, flags)) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nlb = P.NPpad / fbc::line_cols(P.L);
    double* dots = P.d_relax;
    double* gmax = P.d_relax + (size_t)P.opt.max_rhs * fbc::kRelaxBlocks * 2;
    cudaError_t e = cudaSuccess;
    if (f_old) e = fbc::launch_relax_dots(f_new, f_old, (size_t)P.n_i * P.L * 3, n_rhs, dots, st);
    if (e != cudaSuccess) return cuda_fail(e, "relaxation dot products");
    if (int s = apply_modes(P, f_new, n_rhs, flags, st)) return s;
    // ||G f_new||_inf per right-hand side (a pass of the inverse transform that writes nothing)
    if (du_max > 0.0) e = fbc::launch_inverse(P, u, n_rhs, 1.0, 0.0, false, st, nullptr, 0.0, gmax);
    if (e == cudaSuccess) e = fbc::launch_relax_alpha(dots, f_old ? 1 : 0, gmax, nlb, n_rhs, du_max, alpha_io, st);
    if (e != cudaSuccess) return cuda_fail(e, "relaxation parameter");
    // u <- u - alpha_{k+1} G f_new, then the optional zero mean
    e = fbc::launch_inverse(P, u, n_rhs, 0.0, 1.0, (flags & FBC_APPLY_ZERO_MEAN_U) != 0, st, alpha_io,
                            -1.0 / (double)P.L, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "inverse transform");
    return FBC_OK;
}

int fbc_apply_host(fbc_plan* plan, const double* f_host, double* u_host, int32_t n_rhs, double alpha, double beta,
                   uint32_t flags, void* stream) {
    g_last_error.clear();
    if (!plan) return fail(FBC_ERR_INVALID_ARG, "plan is NULL");
    fbc::Plan& P = plan->p;
    if (P.host_only) return fail(FBC_ERR_INVALID_ARG, "host-only plan");
    if (!f_host || !u_host) return fail(FBC_ERR_INVALID_ARG, "f or u is NULL");
    if (n_rhs < 1 || n_rhs > P.opt.max_rhs)
        return fail(FBC_ERR_INVALID_ARG, "n_rhs = %d outside [1, max_rhs = %d]", n_rhs, P.opt.max_rhs);
    cudaStream_t st = (cudaStream_t)stream;
    size_t acc = 0;
    if (!P.d_stage_f) {
        int s = dev_alloc(&P.d_stage_f, (size_t)P.opt.max_rhs * P.n_i * P.L * 3, acc, "stage_f");
        if (s) return s;
    }
    if (!P.d_stage_u) {
        int s = dev_alloc(&P.d_stage_u, (size_t)P.opt.max_rhs * P.n_p * P.L * 3, acc, "stage_u");
        if (s) return s;
    }
    P.workspace_bytes += acc;
    if (!P.host_st[0]) {
        for (auto& h : P.host_st) FBC_CUDA(cudaStreamCreateWithFlags(&h, cudaStreamNonBlocking));
        for (auto& e : P.host_ev) FBC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    // The right-hand sides go through in chunks (at least gran each, at most kHostChunks):
    // chunk c is copied in on one stream, applied on the caller's stream once it has arrived, and
    // copied out on a third stream once applied, so copies overlap the applies of other chunks.
    // Each right-hand side is computed as in one apply of all of them.
    // A chunk holds whole right-hand-side groups of the tensor-core forms (their CTAs compute a group's
    // width whatever its fill).
    const int gran = P.precision == FBC_PREC_BF16X6  ? fbc::contract_oz_rhs_group()
                     : fbc::is_tensor_precision(P.precision) ? fbc::contract_tc_max_rpc(P)
                                                             : fbc::kHostChunkRhs;
    const int n_chunks = std::max(1, std::min(fbc::kHostChunks, n_rhs / gran));
    int per = (n_rhs + n_chunks - 1) / n_chunks;
    if (gran > fbc::kHostChunkRhs) per = (per + gran - 1) / gran * gran;
    const size_t fr = (size_t)P.n_i * P.L * 3, ur = (size_t)P.n_p * P.L * 3;  // doubles per right-hand side
    cudaStream_t cin = P.host_st[0], cout = P.host_st[1];
    cudaEvent_t* ev = P.host_ev;  // [0] start, [1 + c] chunk c in, [1 + kHostChunks + c] chunk c applied, [last] end
    cudaEvent_t ev_end = ev[2 * fbc::kHostChunks + 1];
    int s = FBC_OK;
    cudaError_t e = cudaEventRecord(ev[0], st);  // after the work already queued on the caller's stream
    if (!e) e = cudaStreamWaitEvent(cin, ev[0], 0);
    if (!e) e = cudaStreamWaitEvent(cout, ev[0], 0);
    for (int c = 0; c < n_chunks && !e; c++) {
        const int r0 = c * per, nr = std::min(per, n_rhs - r0);
        if (nr <= 0) break;
        e = cudaMemcpyAsync(P.d_stage_f + r0 * fr, f_host + r0 * fr, nr * fr * sizeof(double), cudaMemcpyHostToDevice,
                            cin);
        if (!e && beta != 0.0)
            e = cudaMemcpyAsync(P.d_stage_u + r0 * ur, u_host + r0 * ur, nr * ur * sizeof(double),
                                cudaMemcpyHostToDevice, cin);
        if (!e) e = cudaEventRecord(ev[1 + c], cin);
    }
    for (int c = 0; c < n_chunks && !e && !s; c++) {
        const int r0 = c * per, nr = std::min(per, n_rhs - r0);
        if (nr <= 0) break;
        if ((e = cudaStreamWaitEvent(st, ev[1 + c], 0))) break;
        if ((s = apply_common(P, P.d_stage_f + r0 * fr, P.d_stage_u + r0 * ur, nr, alpha, beta, flags, st))) break;
        if ((e = cudaEventRecord(ev[1 + fbc::kHostChunks + c], st))) break;
        if ((e = cudaStreamWaitEvent(cout, ev[1 + fbc::kHostChunks + c], 0))) break;
        e = cudaMemcpyAsync(u_host + r0 * ur, P.d_stage_u + r0 * ur, nr * ur * sizeof(double), cudaMemcpyDeviceToHost,
                            cout);
    }
    if (!e && !s) e = cudaEventRecord(ev_end, cout);
    if (!e && !s) e = cudaStreamWaitEvent(st, ev_end, 0);  // the caller's stream ends after the last copy out
    // the host buffers stay in use until every copy has finished, on the error paths too
    const cudaError_t e_in = cudaStreamSynchronize(cin), e_out = cudaStreamSynchronize(cout);
    const cudaError_t e_st = cudaStreamSynchronize(st);
    if (s) return s;
    if (!e) e = e_in ? e_in : (e_out ? e_out : e_st);
    if (e) return cuda_fail(e, "host-memory apply");
    return FBC_OK;
}

int fbc_plan_set_wait_limit(fbc_plan* plan, int32_t polls) {
    g_last_error.clear();
    if (!plan) return fail(FBC_ERR_INVALID_ARG, "plan is NULL");
    if (polls < 0 || polls > (1 << 24)) return fail(FBC_ERR_INVALID_ARG, "polls must be in [0, 2^24]");
    plan->p.wait_limit = polls;
    return FBC_OK;
}

int fbc_plan_set_timing(fbc_plan* plan, int32_t enable) {
    g_last_error.clear();
    if (!plan) return fail(FBC_ERR_INVALID_ARG, "plan is NULL");
    fbc::Plan& P = plan->p;
    if (P.host_only) return fail(FBC_ERR_INVALID_ARG, "host-only plan");
    if (enable && !P.ev[0])
        for (auto& e : P.ev) FBC_CUDA(cudaEventCreate(&e));
    P.timing = enable != 0;
    P.timed_once = false;
    return FBC_OK;
}

int fbc_plan_stage_times(fbc_plan* plan, float* ms) {
    g_last_error.clear();
    if (!plan || !ms) return fail(FBC_ERR_INVALID_ARG, "plan or ms is NULL");
    fbc::Plan& P = plan->p;
    if (!P.timed_once) return fail(FBC_ERR_INVALID_ARG, "no timed apply since timing was enabled");
    FBC_CUDA(cudaEventSynchronize(P.ev[3]));
    for (int t = 0; t < 3; t++) FBC_CUDA(cudaEventElapsedTime(&ms[t], P.ev[t], P.ev[t + 1]));
    return FBC_OK;
}

int fbc_plan_info_get(const fbc_plan* plan, fbc_plan_info* info) {
    g_last_error.clear();
    if (!plan || !info) return fail(FBC_ERR_INVALID_ARG, "plan or info is NULL");
    const fbc::Plan& P = plan->p;
    info->n_i = P.n_i, info->n_p = P.n_p, info->L = P.L, info->K = P.K;
    info->max_rhs = P.opt.max_rhs, info->precision = P.precision;
    info->tile_a = P.TA, info->tile_b = P.TB, info->n_tiles_a = P.n_ta, info->n_tiles_b = P.n_tb;
    info->box_x0 = P.box_x0, info->box_y0 = P.box_y0, info->box_nx = P.Dx, info->box_ny = P.Dy;
    info->sub_w = P.W, info->sub_h = P.H, info->n_used_d = P.n_used;
    info->tabulated = P.tabulated ? 1 : 0;
    info->pair_modes_per_rhs = (double)P.n_p * (double)P.n_i * (double)P.K;
    info->table_bytes = P.table_bytes;
    info->surrogate_bytes = P.sur_bytes;
    info->surrogate_attached = P.sur ? 1 : 0;
    info->n_far_d = P.n_far;
    info->surrogate_chunk = P.sur_chunk;
    info->reserved = 0;
    fbc::fft_info(P, &info->fft_mx, &info->fft_my, &info->fft_rows_i, &info->fft_rows_p, &info->fft_chunk_items);
    info->reserved2 = 0;
    info->workspace_bytes = P.workspace_bytes;
    return FBC_OK;
}

int fbc_plan_layout(const fbc_plan* plan, int32_t* perm_i, int32_t* perm_p, int32_t* xy_i, int32_t* xy_p) {
    g_last_error.clear();
    if (!plan) return fail(FBC_ERR_INVALID_ARG, "plan is NULL");
    const fbc::Plan& P = plan->p;
    for (int s = 0; s < P.NIpad; s++) {
        if (perm_i) perm_i[s] = P.perm_i[s];
        if (xy_i) xy_i[2 * s] = P.xy_i_sorted[s].x, xy_i[2 * s + 1] = P.xy_i_sorted[s].y;
    }
    for (int s = 0; s < P.NPpad; s++) {
        if (perm_p) perm_p[s] = P.perm_p[s];
        if (xy_p) xy_p[2 * s] = P.xy_p_sorted[s].x, xy_p[2 * s + 1] = P.xy_p_sorted[s].y;
    }
    return FBC_OK;
}

int fbc_get_mode_table(const fbc_plan* plan, const int32_t* d, int32_t nd, double* out) {
    g_last_error.clear();
    if (!plan || (!d && nd) || (!out && nd) || nd < 0) return fail(FBC_ERR_INVALID_ARG, "bad arguments");
    const fbc::Plan& P = plan->p;
    if (P.host_only) return fail(FBC_ERR_INVALID_ARG, "host-only plan");
    if (!P.tabulated) return fail(FBC_ERR_NOT_TABULATED, "table not tabulated");
    if (!P.d_table) return fail(FBC_ERR_UNSUPPORTED, "the plan's tables were released for its surrogate");
    FBC_CUDA(cudaDeviceSynchronize());
    for (int t = 0; t < nd; t++) {
        int ix = d[2 * t] - P.box_x0, iy = d[2 * t + 1] - P.box_y0;
        if (ix < 0 || ix >= P.Dx || iy < 0 || iy >= P.Dy)
            return fail(FBC_ERR_INVALID_ARG, "difference (%d, %d) outside the table box", d[2 * t], d[2 * t + 1]);
        for (int k = 0; k < P.K; k++) {
            const double* src = P.d_table + (((size_t)k * P.Dy + iy) * P.Dx + ix) * 6;
            FBC_CUDA(cudaMemcpy(out + ((size_t)t * P.K + k) * 6, src, 6 * sizeof(double), cudaMemcpyDeviceToHost));
        }
    }
    return FBC_OK;
}

int fbc_plan_sync_status(fbc_plan* plan, void* stream) {
    g_last_error.clear();
    if (!plan) return fail(FBC_ERR_INVALID_ARG, "plan is NULL");
    fbc::Plan& P = plan->p;
    if (P.host_only) return fail(FBC_ERR_INVALID_ARG, "host-only plan");
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    FBC_CUDA(cudaMemcpyAsync(&h, P.d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    FBC_CUDA(cudaStreamSynchronize(st));
    if (h != 0) {
        FBC_CUDA(cudaMemsetAsync(P.d_status, 0, sizeof(int), st));
        FBC_CUDA(cudaStreamSynchronize(st));
        return fail(FBC_ERR_TIMEOUT, "device status word %d", h);
    }
    return FBC_OK;
}

void fbc_destroy(fbc_plan* plan) {
    if (!plan) return;
    if (!plan->p.host_only) cudaDeviceSynchronize();
    free_plan(plan->p);
    delete plan;
}

}  // extern "C"
