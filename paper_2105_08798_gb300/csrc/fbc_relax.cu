// Residual-based relaxation of the FBC update (Sec. 2.3.3, Algorithm 2),
// computed on the device so that the relaxed update needs no host round trip:
//   alpha_{k+1} = -alpha_k <f_k, f_{k+1} - f_k> / ||f_{k+1} - f_k||^2,
//   alpha_{k+1} = 1 where that is negative,
//   alpha_{k+1} = du_max / ||G f_{k+1}||_inf where ||alpha_{k+1} G f_{k+1}||_inf > du_max.
// One value per right-hand side (each is its own relaxation sequence).  The dot
// products are summed in a fixed order (per-block partials, then one thread),
// so the result does not depend on scheduling.
#include "fbc_internal.cuh"

namespace fbc {
namespace {

// part[r][blk] = (sum f_old (f_new - f_old), sum (f_new - f_old)^2) over block blk's
// strided share of right-hand side r's n elements
__global__ void k_relax_dots(const double* __restrict__ f_new, const double* __restrict__ f_old, size_t n,
                             double* __restrict__ part) {
    __shared__ double rd[256], rn[256];
    const int r = blockIdx.y;
    const double* a = f_new + (size_t)r * n;
    const double* b = f_old + (size_t)r * n;
    double d = 0.0, q = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double df = a[i] - b[i];
        d = fma(b[i], df, d);
        q = fma(df, df, q);
    }
    rd[threadIdx.x] = d, rn[threadIdx.x] = q;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) rd[threadIdx.x] += rd[threadIdx.x + w], rn[threadIdx.x] += rn[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* p = part + ((size_t)r * gridDim.x + blockIdx.x) * 2;
        p[0] = rd[0], p[1] = rn[0];
    }
}

// One thread per right-hand side: Algorithm 2.  With equal f_new and f_old (a zero
// denominator) alpha_k is kept.
__global__ void k_relax_alpha(const double* __restrict__ dot_part, int has_old, const double* __restrict__ gmax_part,
                              int n_gblk, int n_rhs, double du_max, double* __restrict__ alpha_io) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rhs) return;
    double alpha = alpha_io[r];
    if (has_old) {
        double d = 0.0, q = 0.0;
        for (int b = 0; b < kRelaxBlocks; b++) {
            d += dot_part[((size_t)r * kRelaxBlocks + b) * 2];
            q += dot_part[((size_t)r * kRelaxBlocks + b) * 2 + 1];
        }
        if (q > 0.0) alpha = -alpha * d / q;
        if (alpha < 0.0) alpha = 1.0;
    }
    if (du_max > 0.0) {
        double gmax = 0.0;
        for (int b = 0; b < n_gblk; b++) gmax = fmax(gmax, gmax_part[(size_t)r * n_gblk + b]);
        if (gmax > 0.0 && alpha * gmax > du_max) alpha = du_max / gmax;
    }
    alpha_io[r] = alpha;
}

}  // namespace

cudaError_t launch_relax_dots(const double* f_new, const double* f_old, size_t n_per_rhs, int n_rhs, double* part,
                              cudaStream_t st) {
    k_relax_dots<<<dim3(kRelaxBlocks, n_rhs), 256, 0, st>>>(f_new, f_old, n_per_rhs, part);
    return cudaGetLastError();
}

cudaError_t launch_relax_alpha(const double* dot_part, int has_old, const double* gmax_part, int n_gblk, int n_rhs,
                               double du_max, double* alpha_io, cudaStream_t st) {
    k_relax_alpha<<<(n_rhs + 63) / 64, 64, 0, st>>>(dot_part, has_old, gmax_part, n_gblk, n_rhs, du_max, alpha_io);
    return cudaGetLastError();
}

}  // namespace fbc
