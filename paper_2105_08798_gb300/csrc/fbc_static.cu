// Allocation-free zero-mean step for callers that cannot allocate device memory.
//
// Some callers of the pad update cannot call cudaMalloc at the point where
// they want to re-centre the pad displacements: an atomistic engine that has
// handed the whole device to its own memory pool, or a tight relaxation loop
// that must not take the allocator's device-wide lock.
// fbc_zero_mean_static() gives them the zero-mean step (subtract, per
// right-hand side and component, the mean displacement over all n_p * L pad
// atoms) with its reduction scratch in a fixed array of this library, so the
// call itself allocates nothing.
//
// The scratch is g_zero_mean_scratch below: kStaticMaxRhs * kStaticBlocks * 3
// doubles (384 KiB).  Every GPU that loads the library holds it until the
// process exits.  All calls share it and it keeps the last call's contents;
// each call writes every slot it later reads, so nothing has to start at zero.
// Calls that overlap on the GPU (different streams, or different host threads
// without ordering) race on it.
//
// Host code must not pass the array's name to a kernel: on the host it is only
// a stand-in symbol.  Its device address comes from cudaGetSymbolAddress with
// the device current.  The first call on a device looks it up (make that call
// before any stream capture); later calls made outside a stream capture look
// it up again, so that a cudaDeviceReset, after which the module is loaded
// anew and the array may move, is followed by one such call before the next
// capture.  A call made while its stream is being captured uses the address of
// the last lookup on that device.
#include <mutex>

#include "fbc_internal.cuh"

namespace {

constexpr int kStaticMaxRhs = 64;
constexpr int kStaticBlocks = 256;
constexpr int kStaticThreads = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_zero_mean_scratch[kStaticMaxRhs * kStaticBlocks * 3];

// Pass 1: block b of right-hand side r sums a strided share of u[r] per component.
__global__ void k_static_partials(const double* __restrict__ u, double* __restrict__ scratch, size_t n_atoms) {
    __shared__ double red[3][kStaticThreads];
    const int r = blockIdx.y;
    const double* ur = u + (size_t)r * n_atoms * 3;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_atoms; i += (size_t)gridDim.x * blockDim.x) {
        s0 += ur[3 * i];
        s1 += ur[3 * i + 1];
        s2 += ur[3 * i + 2];
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    for (int w = kStaticThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int c = 0; c < 3; c++) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* o = scratch + ((size_t)r * gridDim.x + blockIdx.x) * 3;
        o[0] = red[0][0], o[1] = red[1][0], o[2] = red[2][0];
    }
}

// Pass 2: every block reduces the partials of its right-hand side in the same
// fixed order (deterministic) and subtracts the mean from its share of u[r].
__global__ void k_static_subtract(double* __restrict__ u, const double* __restrict__ scratch, int n_part,
                                  size_t n_atoms) {
    __shared__ double mean[3];
    const int r = blockIdx.y;
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        const double* p = scratch + (size_t)r * n_part * 3;
        for (int t = 0; t < n_part; t++) s0 += p[3 * t], s1 += p[3 * t + 1], s2 += p[3 * t + 2];
        const double inv = 1.0 / (double)n_atoms;
        mean[0] = s0 * inv, mean[1] = s1 * inv, mean[2] = s2 * inv;
    }
    __syncthreads();
    double* ur = u + (size_t)r * n_atoms * 3;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_atoms * 3; i += (size_t)gridDim.x * blockDim.x)
        ur[i] -= mean[i % 3];
}

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};

int static_fail(int code, const char* msg) { return fbc::report_error(code, msg); }

}  // namespace

extern "C" {

int fbc_zero_mean_static(double* u, int32_t n_rhs, int32_t n_p, int32_t L, void* stream) {
    fbc::report_error(FBC_OK, "");
    if (!u) return static_fail(FBC_ERR_INVALID_ARG, "u is NULL");
    if (n_p < 1 || L < 1) return static_fail(FBC_ERR_INVALID_ARG, "n_p and L must be >= 1");
    if (n_rhs < 1 || n_rhs > kStaticMaxRhs)
        return static_fail(FBC_ERR_INVALID_ARG,
                           "n_rhs must be in [1, 64]: the fixed scratch holds 64 right-hand sides");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return static_fail(FBC_ERR_CUDA, "cudaGetDevice failed or device index out of range");
    cudaStream_t st = (cudaStream_t)stream;
    // outside a capture the address is looked up afresh (it may have moved after a device reset)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone;
    if (capturing) cudaGetLastError();  // a failed query leaves no sticky error
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_addr_mu);
        if (!g_addr[dev] || !capturing) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_zero_mean_scratch);
            if (e != cudaSuccess || !p) return static_fail(FBC_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed");
            g_addr[dev] = p;
        }
        scratch = g_addr[dev];
    }
    const size_t n_atoms = (size_t)n_p * (size_t)L;
    dim3 grid(kStaticBlocks, n_rhs);
    k_static_partials<<<grid, kStaticThreads, 0, st>>>(u, (double*)scratch, n_atoms);
    if (cudaGetLastError() != cudaSuccess) return static_fail(FBC_ERR_CUDA, "launch of the partial sums failed");
    k_static_subtract<<<grid, kStaticThreads, 0, st>>>(u, (const double*)scratch, kStaticBlocks, n_atoms);
    if (cudaGetLastError() != cudaSuccess) return static_fail(FBC_ERR_CUDA, "launch of the subtraction failed");
    return FBC_OK;
}

}  // extern "C"
