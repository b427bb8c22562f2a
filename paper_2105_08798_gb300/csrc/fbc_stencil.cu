// Incompatibility force of the FBC iteration (Sec. 2.3.2, Eq. 21; the step after
// the atomistic solve in Algorithm 1):
//   f_in(a) = L_h^{i+|i}[u_{k+1}](a) + L_h^{i+|i++}[u_k](a),   a in Lambda^{i+},
// i.e. the harmonic operator L_h, restricted to the rows of the interface
// columns, applied to a displacement field assembled from several site sets
// (the relaxed atoms with their new displacements, the continuum nodes with
// the previous ones).  L_h is local: a 27-point block stencil on the
// line-periodic lattice,
//   L_h[u](x, q) = sum_{n in {-1,0,1}^3} K(n) u(x + (n_x, n_y), (q + n_z) mod L),
// with K(n) a real 3x3 block (the force-constant tensor of the harmonic model).
//
// Host side: the neighbour table of every interface column (for each of the 9
// in-plane offsets, the source set and column that holds the site) is built
// once with a hash map of the sites.  Device side: one thread per (rhs,
// interface column, plane) gathers the 27 neighbours it needs (3 doubles each,
// consecutive planes in consecutive threads) and accumulates K(n) u in FP64.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <unordered_map>
#include <vector>

#include "fbc_internal.cuh"

struct fbc_stencil {
    int n_i = 0, L = 0, n_src = 0;
    int n_site[FBC_STENCIL_MAX_SOURCES] = {0, 0, 0, 0};
    unsigned mask = 0;     // bit j: K(offset j) is not all zero
    int* d_nbr = nullptr;  // [n_i][9] (source << 28) | column, -1 = not needed
    double* d_K = nullptr; // [27][9]
};

namespace {

constexpr int kSrcShift = 28;
constexpr int kColMask = (1 << kSrcShift) - 1;

int st_fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return fbc::report_error(code, buf);
}

struct StencilArgs {
    const int* nbr;
    const double* K;
    const double* u[FBC_STENCIL_MAX_SOURCES];
    long long u_rhs_stride[FBC_STENCIL_MAX_SOURCES];  // n_site[s] * L * 3
    double* f;
    int n_i, L, n_rhs;
    unsigned mask;
};

__global__ void __launch_bounds__(256) k_incompat(StencilArgs A) {
    __shared__ double sK[27 * 9];
    for (int t = threadIdx.x; t < 27 * 9; t += blockDim.x) sK[t] = A.K[t];
    __syncthreads();
    const long long n_el = (long long)A.n_rhs * A.n_i * A.L;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const int q = (int)(e % A.L);
    const long long ra = e / A.L;
    const int a = (int)(ra % A.n_i);
    const int r = (int)(ra / A.n_i);
    double f0 = 0.0, f1 = 0.0, f2 = 0.0;
    for (int c = 0; c < 9; c++) {  // in-plane offset (dx, dy) = (c / 3 - 1, c % 3 - 1)
        if (!((A.mask >> (3 * c)) & 7u)) continue;
        const int code = __ldg(A.nbr + (size_t)a * 9 + c);
        const int s = code >> kSrcShift;
        // selects rather than a dynamic index, which would copy the parameter block to local memory
        const double* base = s == 0 ? A.u[0] : s == 1 ? A.u[1] : s == 2 ? A.u[2] : A.u[3];
        const long long stride = s == 0   ? A.u_rhs_stride[0]
                                 : s == 1 ? A.u_rhs_stride[1]
                                 : s == 2 ? A.u_rhs_stride[2]
                                          : A.u_rhs_stride[3];
        const double* col = base + r * stride + (long long)(code & kColMask) * A.L * 3;
        for (int dz = 0; dz < 3; dz++) {
            const int j = 3 * c + dz;
            if (!((A.mask >> j) & 1u)) continue;
            int p = q + dz - 1;
            p = p < 0 ? p + A.L : (p >= A.L ? p - A.L : p);
            const double u0 = col[3 * p], u1 = col[3 * p + 1], u2 = col[3 * p + 2];
            const double* k = sK + 9 * j;
            f0 = fma(k[0], u0, fma(k[1], u1, fma(k[2], u2, f0)));
            f1 = fma(k[3], u0, fma(k[4], u1, fma(k[5], u2, f1)));
            f2 = fma(k[6], u0, fma(k[7], u1, fma(k[8], u2, f2)));
        }
    }
    double* o = A.f + e * 3;
    o[0] = f0, o[1] = f1, o[2] = f2;
}

inline unsigned long long site_key(int x, int y) {
    return ((unsigned long long)(unsigned)x << 32) | (unsigned)y;
}

}  // namespace

extern "C" {

int fbc_spring_constants(double k1, double k2, double c, double* K) {
    fbc::report_error(FBC_OK, "");
    if (!K) return st_fail(FBC_ERR_INVALID_ARG, "K is NULL");
    if (!std::isfinite(k1) || !std::isfinite(k2) || !(c > 0.0) || !std::isfinite(c))
        return st_fail(FBC_ERR_INVALID_ARG, "k1, k2 must be finite and c > 0");
    std::memset(K, 0, sizeof(double) * 27 * 9);
    double* K0 = K + 9 * 13;
    for (int nx = -1; nx <= 1; nx++)
        for (int ny = -1; ny <= 1; ny++)
            for (int nz = -1; nz <= 1; nz++) {
                const int l1 = std::abs(nx) + std::abs(ny) + std::abs(nz);
                if (l1 == 0 || l1 == 3) continue;
                const double k = l1 == 1 ? k1 : k2;
                const double v[3] = {(double)nx, (double)ny, nz * c};
                const double n2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                double* Kn = K + 9 * ((nx + 1) * 9 + (ny + 1) * 3 + (nz + 1));
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) {
                        const double b = k * v[i] * v[j] / n2;
                        Kn[3 * i + j] = -b;
                        K0[3 * i + j] += b;
                    }
            }
    return FBC_OK;
}

int fbc_stencil_create(int32_t n_i, const int32_t* xy_i, int32_t n_src, const int32_t* const* xy_src,
                       const int32_t* n_site, int32_t L, const double* K, fbc_stencil** out) {
    fbc::report_error(FBC_OK, "");
    if (!out) return st_fail(FBC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_i < 1 || !xy_i) return st_fail(FBC_ERR_INVALID_ARG, "need n_i >= 1 interface sites");
    if (L < 1) return st_fail(FBC_ERR_INVALID_ARG, "L must be >= 1");
    if (n_src < 1 || n_src > FBC_STENCIL_MAX_SOURCES || !xy_src || !n_site)
        return st_fail(FBC_ERR_INVALID_ARG, "n_src must be in [1, %d]", FBC_STENCIL_MAX_SOURCES);
    if (!K) return st_fail(FBC_ERR_INVALID_ARG, "K is NULL");
    unsigned mask = 0;
    for (int j = 0; j < 27; j++) {
        for (int t = 0; t < 9; t++) {
            if (!std::isfinite(K[9 * j + t])) return st_fail(FBC_ERR_INVALID_ARG, "K has a non-finite entry");
            if (K[9 * j + t] != 0.0) mask |= 1u << j;
        }
    }
    std::unordered_map<unsigned long long, int> where;
    size_t total = 0;
    for (int s = 0; s < n_src; s++) {
        if (n_site[s] < 0 || n_site[s] > kColMask || (n_site[s] > 0 && !xy_src[s]))
            return st_fail(FBC_ERR_INVALID_ARG, "source %d: bad site count or NULL sites", s);
        total += (size_t)n_site[s];
    }
    where.reserve(total * 2);
    for (int s = 0; s < n_src; s++)
        for (int t = 0; t < n_site[s]; t++) {
            const int x = xy_src[s][2 * t], y = xy_src[s][2 * t + 1];
            auto ins = where.emplace(site_key(x, y), (s << kSrcShift) | t);
            if (!ins.second)
                return st_fail(FBC_ERR_INVALID_ARG, "site (%d, %d) appears twice in the source sets", x, y);
        }
    std::vector<int> nbr((size_t)n_i * 9, -1);
    for (int a = 0; a < n_i; a++)
        for (int c = 0; c < 9; c++) {
            if (!((mask >> (3 * c)) & 7u)) continue;
            const int x = xy_i[2 * a] + c / 3 - 1, y = xy_i[2 * a + 1] + c % 3 - 1;
            auto it = where.find(site_key(x, y));
            if (it == where.end())
                return st_fail(FBC_ERR_INVALID_ARG,
                               "site (%d, %d), a neighbour of interface column %d, is in no source set", x, y, a);
            nbr[(size_t)a * 9 + c] = it->second;
        }
    fbc_stencil* S = new (std::nothrow) fbc_stencil();
    if (!S) return st_fail(FBC_ERR_OOM, "host allocation failed");
    S->n_i = n_i, S->L = L, S->n_src = n_src, S->mask = mask;
    for (int s = 0; s < n_src; s++) S->n_site[s] = n_site[s];
    cudaError_t e = cudaMalloc((void**)&S->d_nbr, sizeof(int) * nbr.size());
    if (!e) e = cudaMalloc((void**)&S->d_K, sizeof(double) * 27 * 9);
    if (!e) e = cudaMemcpy(S->d_nbr, nbr.data(), sizeof(int) * nbr.size(), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(S->d_K, K, sizeof(double) * 27 * 9, cudaMemcpyHostToDevice);
    if (e) {
        fbc_stencil_destroy(S);
        return st_fail(e == cudaErrorMemoryAllocation ? FBC_ERR_OOM : FBC_ERR_CUDA, "stencil upload: %s",
                       cudaGetErrorString(e));
    }
    *out = S;
    return FBC_OK;
}

int fbc_incompat_force(const fbc_stencil* st, const double* const* u_src, double* f_in, int32_t n_rhs,
                       void* stream) {
    fbc::report_error(FBC_OK, "");
    if (!st) return st_fail(FBC_ERR_INVALID_ARG, "stencil is NULL");
    if (!u_src || !f_in) return st_fail(FBC_ERR_INVALID_ARG, "u_src or f_in is NULL");
    if (n_rhs < 1) return st_fail(FBC_ERR_INVALID_ARG, "n_rhs must be >= 1");
    StencilArgs A{};
    A.nbr = st->d_nbr, A.K = st->d_K, A.f = f_in;
    A.n_i = st->n_i, A.L = st->L, A.n_rhs = n_rhs, A.mask = st->mask;
    for (int s = 0; s < st->n_src; s++) {
        if (!u_src[s] && st->n_site[s] > 0) return st_fail(FBC_ERR_INVALID_ARG, "u_src[%d] is NULL", s);
        A.u[s] = u_src[s];
        A.u_rhs_stride[s] = (long long)st->n_site[s] * st->L * 3;
    }
    const long long n_el = (long long)n_rhs * st->n_i * st->L;
    const long long blocks = (n_el + 255) / 256;
    if (blocks > 0x7fffffffLL) return st_fail(FBC_ERR_INVALID_ARG, "problem too large for one launch");
    k_incompat<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(A);
    const cudaError_t e = cudaGetLastError();
    if (e) return st_fail(FBC_ERR_CUDA, "incompatibility force launch: %s", cudaGetErrorString(e));
    return FBC_OK;
}

int fbc_stencil_destroy(fbc_stencil* st) {
    if (!st) return FBC_OK;
    if (st->d_nbr) cudaFree(st->d_nbr);
    if (st->d_K) cudaFree(st->d_K);
    delete st;
    return FBC_OK;
}

}  // extern "C"
