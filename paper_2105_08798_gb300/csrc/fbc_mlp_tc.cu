// Fused inference of the mode-table surrogate on the tensor cores (tcgen05).
//
// One CTA (8 warps) walks tiles of 128 rows; for each tile the whole network
// 4 -> H -> H -> H -> 6 runs without leaving the SM:
//   * the row features (computed from the difference and the mode, or read)
//     are split into three bf16 pieces and stored as the A operand [128][16];
//   * each layer is one or two passes of tcgen05.mma (M = 128, N = H or 16,
//     K = 16 per instruction) over the activation pieces, against the layer's
//     BF16 weights held in shared memory for the kernel's lifetime, with the
//     FP32 accumulator in tensor memory;
//   * the epilogue reads the accumulator (tcgen05.ld), adds the bias, applies
//     SiLU and splits the activation into hi + lo bf16 pieces for the next
//     layer (warps w and w + 4 share a TMEM lane quadrant and take one half of
//     the columns each);
//   * the last layer's six outputs are written as rows, or multiplied by the
//     decay s(q, r) and written straight into the mode slice of the difference.
// Weights are exact in bf16 and activations carry about 16 mantissa bits
// (inputs 24), so the result matches an FP32 evaluation with BF16 weights to
// a few units in 1e-5.
//
// Every wait on the mbarrier is bounded; on a timeout the CTA records the
// status word, stops, waits once more (bounded) for its own tensor-core work,
// frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "fbc_internal.cuh"
#include "fbc_tc.cuh"

namespace fbc {
namespace {

constexpr int kThreads = 256;
constexpr int kRows = 128;
constexpr int kMaxH = 128;
constexpr int kXPieces = 3, kActPieces = 2;
constexpr int kXBytes = kRows * 16 * 2;  // one [128][16] bf16 piece

using tc::canon_bf16;
using tc::mbar_wait;
using tc::sdesc;
using tc::smem_u32;

size_t smem_bytes(int H) {
    return (size_t)H * 16 * 2 + 2 * (size_t)H * H * 2 + (size_t)16 * H * 2 + (size_t)kXPieces * kXBytes +
           (size_t)kActPieces * kRows * H * 2 + (size_t)(3 * H + 16) * 4;
}

__device__ __forceinline__ uint32_t bf16_bits(float x) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x)); }

// 8 consecutive K elements of one row, split into pieces, stored as one
// 16-byte core-matrix row per piece
template <int NP>
__device__ __forceinline__ void store_split8(unsigned char* base, size_t piece_stride, uint32_t off, const float* v) {
    uint32_t w[NP][8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        float r = v[i];
#pragma unroll
        for (int p = 0; p < NP; p++) {
            const __nv_bfloat16 h = __float2bfloat16_rn(r);
            w[p][i] = (uint32_t)__bfloat16_as_ushort(h);
            r = __fsub_rn(r, __bfloat162float(h));
        }
    }
#pragma unroll
    for (int p = 0; p < NP; p++) {
        uint4 q;
        q.x = w[p][0] | (w[p][1] << 16), q.y = w[p][2] | (w[p][3] << 16);
        q.z = w[p][4] | (w[p][5] << 16), q.w = w[p][6] | (w[p][7] << 16);
        *(uint4*)(base + p * piece_stride + off) = q;
    }
}

__device__ __forceinline__ float silu(float z) { return z * __frcp_rn(1.f + expf(-z)); }

template <bool SLICE>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_tc(MlpArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase;
    __shared__ int s_abort;
    const int H = a.H;
    const uint32_t sboH = (uint32_t)H * 16;          // 8-row group stride of a K = H operand
    unsigned char* sW1 = smem;                        // [H][16]
    unsigned char* sW2 = sW1 + (size_t)H * 16 * 2;    // [H][H]
    unsigned char* sW3 = sW2 + (size_t)H * H * 2;     // [H][H]
    unsigned char* sW4 = sW3 + (size_t)H * H * 2;     // [16][H]
    unsigned char* sX = sW4 + (size_t)16 * H * 2;     // 3 x [128][16]
    unsigned char* sAct = sX + kXPieces * kXBytes;    // 2 x [128][H]
    float* sBias = (float*)(sAct + (size_t)kActPieces * kRows * H * 2);  // b1 b2 b3 [H], b4 [16]
    const size_t actPiece = (size_t)kRows * H * 2;

    // weights as B operands [N][K] (element (n, k) = W[k][n]), zero padded
    {
        const float* P = a.params;
        for (int e = threadIdx.x; e < H * 16; e += kThreads) {
            const int kk = e / H, n = e % H;
            const float v = kk < kSurIn ? P[a.off[0] + kk * H + n] : 0.f;
            *(uint16_t*)(sW1 + canon_bf16(n, kk, 256)) = (uint16_t)bf16_bits(v);
        }
        for (int l = 0; l < 2; l++) {
            const float* W = P + a.off[2 + 2 * l];
            unsigned char* dst = l ? sW3 : sW2;
            for (int e = threadIdx.x; e < H * H; e += kThreads) {
                const int kk = e / H, n = e % H;
                *(uint16_t*)(dst + canon_bf16(n, kk, sboH)) = (uint16_t)bf16_bits(W[e]);
            }
        }
        for (int e = threadIdx.x; e < 16 * H; e += kThreads) {
            const int kk = e / 16, n = e % 16;
            const float v = n < kSurOut ? P[a.off[6] + kk * kSurOut + n] : 0.f;
            *(uint16_t*)(sW4 + canon_bf16(n, kk, sboH)) = (uint16_t)bf16_bits(v);
        }
        for (int e = threadIdx.x; e < 3 * H; e += kThreads) sBias[e] = P[a.off[1 + 2 * (e / H)] + e % H];
        for (int e = threadIdx.x; e < 16; e += kThreads) sBias[3 * H + e] = e < kSurOut ? P[a.off[7] + e] : 0.f;
    }
    if (threadIdx.x == 0) {
        s_abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                     "r"(kMaxH));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;                       // TMEM lane = row of the tile
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
    const int tiles_per_mode = (a.n + kRows - 1) / kRows;
    const int n_tiles = tiles_per_mode * (SLICE ? a.n_modes : 1);
    const uint32_t idH = tc::idesc(1, kRows, H), id16 = tc::idesc(1, kRows, 16);
    uint32_t phase = 0;
    bool pending = false;

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int mj = tile / tiles_per_mode;
        const int i = (tile % tiles_per_mode) * kRows + row;
        const bool valid = i < a.n;
        double sc = 0.0;
        size_t cell = 0;
        if (half == 0) {
            float x[16];
#pragma unroll
            for (int j = 0; j < 16; j++) x[j] = 0.f;
            if (valid) {
                if (SLICE) {
                    const int2 d = a.far[i];
                    const double qr = surrogate_features(d.x, d.y, a.k0 + mj, a.L, a.c, x);
                    sc = surrogate_scale(qr, a.c);
                    cell = (size_t)(d.y - a.box_y0) * a.Dx + (d.x - a.box_x0);
                } else {
#pragma unroll
                    for (int j = 0; j < kSurIn; j++) x[j] = a.X[(size_t)i * kSurIn + j];
                }
            }
            store_split8<kXPieces>(sX, kXBytes, canon_bf16(row, 0, 256), x);
            store_split8<kXPieces>(sX, kXBytes, canon_bf16(row, 8, 256), x + 8);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        for (int l = 0; l < 4; l++) {
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (l == 0) {
                    for (int p = 0; p < kXPieces; p++)
                        tc::mma_bf16(tmem, sdesc(smem_u32(sX + p * kXBytes), 128, 256), sdesc(smem_u32(sW1), 128, 256),
                                     idH, p > 0);
                } else {
                    const unsigned char* B = l == 1 ? sW2 : l == 2 ? sW3 : sW4;
                    const uint32_t id = l == 3 ? id16 : idH;
                    for (int p = 0; p < kActPieces; p++)
                        for (int s = 0; s < H / 16; s++)
                            tc::mma_bf16(tmem, sdesc(smem_u32(sAct + p * actPiece) + 256 * s, 128, sboH),
                                         sdesc(smem_u32(B) + 256 * s, 128, sboH), id, (p | s) ? 1u : 0u);
                }
                tc::commit(&mbar);
            }
            const bool ok = mbar_wait(&mbar, phase);
            pending = !ok;
            if (ok) phase ^= 1u;
            else s_abort = 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            __syncthreads();
            if (s_abort) break;
            if (l < 3) {
                const float* bias = sBias + l * H;
                for (int c0 = half * (H / 2); c0 < (half + 1) * (H / 2); c0 += 16) {
                    float v[16];
                    tc::ld16(trow + (uint32_t)c0, v);
#pragma unroll
                    for (int j = 0; j < 16; j++) v[j] = silu(v[j] + bias[c0 + j]);
                    store_split8<kActPieces>(sAct, actPiece, canon_bf16(row, c0, sboH), v);
                    store_split8<kActPieces>(sAct, actPiece, canon_bf16(row, c0 + 8, sboH), v + 8);
                }
            } else if (half == 0) {
                float v[16];
                tc::ld16(trow, v);
                if (valid) {
                    if (SLICE) {
                        float* o = a.slice + (size_t)mj * a.slice_floats + cell * kSurOut;
#pragma unroll
                        for (int j = 0; j < kSurOut; j++) o[j] = (float)((double)(v[j] + sBias[3 * H + j]) * sc);
                    } else {
#pragma unroll
                        for (int j = 0; j < kSurOut; j++) a.Y[(size_t)i * kSurOut + j] = v[j] + sBias[3 * H + j];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
        if (s_abort) break;
    }
    if (s_abort) {
        if (threadIdx.x == 0) atomicExch(a.status, FBC_ERR_TIMEOUT);
        // second and last bounded wait for this CTA's own tensor-core work
        if (pending) mbar_wait(&mbar, phase);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMaxH));
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    }
    return n;
}

}  // namespace

// the epilogue gives each half of the CTA H / 2 columns in steps of 16
bool mlp_tc_supported(int H) { return H >= 32 && H <= kMaxH && H % 32 == 0; }

cudaError_t launch_mlp_tc(const MlpArgs& a, cudaStream_t st) {
    if (!mlp_tc_supported(a.H) || a.n < 1 || !a.status) return cudaErrorInvalidValue;
    const size_t smem = smem_bytes(a.H);
    const int tiles = ((a.n + kRows - 1) / kRows) * (a.slice ? a.n_modes : 1);
    const int grid = std::min(tiles, sm_count());
    if (a.slice) {
        if (!a.far || a.n_modes < 1) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e) return e;
        k_mlp_tc<true><<<grid, kThreads, smem, st>>>(a);
    } else {
        if (!a.X || !a.Y) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e) return e;
        k_mlp_tc<false><<<grid, kThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace fbc
