// Per-mode contraction on the 5th-generation tensor cores (tcgen05, FP32
// accumulation in tensor memory), for plans with several right-hand sides.
//
// For one wavenumber k the update is a real GEMM (Sec. 3.2, Eqs. 37-38 in the
// mode domain): with the six-vector form, every pad column a and output
// component c receives
//     U_c(a, :) = sum_{c', b} M_{c c'}(x_a - x_b) X_{c'}(b, :),
// where the columns ':' are the x and y' halves of all right-hand sides and
// M = [[A11, A12, -B13], [A12, A22, -B23], [B13, B23, A33]] comes from the six
// table reals.  A CTA owns 128 pad columns (GEMM rows) at one k and up to 64
// right-hand sides (N = 2 R columns); it walks the interface tiles in steps
// of KB columns, and for each step
//   * gathers the six 128 x KB blocks A_e(a, b) = T_e(x_a - x_b) from the
//     staged table sub-box and splits them into bf16 pieces (h, m, l) or
//     rounds them to tf32, written in the K-major no-swizzle canonical layout
//     (8-row x 16-byte core matrices);
//   * converts the transformed forces X_0, X_1, X_2 and -X_2 (the sign of the
//     13/23 entries is carried by this negated copy) the same way;
//   * one thread issues the 9 block products per split-product pair with
//     tcgen05.mma (M = 128, N = 2 R, K = 16 bf16 / 8 tf32) into three TMEM
//     accumulators (one per output component) and commits to an mbarrier.
// Split products: TF32 (1), BF16X2 (hh + hm + mh), BF16X3 (+ hl + lh + mm),
// pieces h = bf16(x), m = bf16(x - h), l = bf16(x - h - m), all rounded to
// nearest.  The logarithmic k = 0 mode is left to the FP64 kernel.
//
// Every wait on the mbarrier is bounded; when a bound is hit the CTA records
// the status word, stops issuing work, waits once more (bounded) for its own
// tensor-core work, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "fbc_internal.cuh"
#include "fbc_tc.cuh"

namespace fbc {
namespace {

constexpr int kTmemCols = 512;
constexpr int kMaxNP = 128;      // 64 right-hand sides x (x, y')
constexpr int kRhsPerCta = 64;
using tc::idesc;
using tc::mbar_wait;
using tc::sdesc;
using tc::smem_u32;

template <int PREC>
struct TcCfg;
template <>
struct TcCfg<FBC_PREC_TF32> {
    static constexpr int ES = 4, NS = 1, NPROD = 1, KB = 32, KMMA = 8, FMT = 2;
};
template <>
struct TcCfg<FBC_PREC_BF16X2> {
    static constexpr int ES = 2, NS = 2, NPROD = 3, KB = 32, KMMA = 16, FMT = 1;
};
template <>
struct TcCfg<FBC_PREC_BF16X3> {
    static constexpr int ES = 2, NS = 3, NPROD = 6, KB = 16, KMMA = 16, FMT = 1;
};

// (piece of A, piece of B) for each split product, by decreasing magnitude
__constant__ int c_prod_a[6] = {0, 0, 1, 0, 2, 1};
__constant__ int c_prod_b[6] = {0, 1, 0, 2, 0, 1};
// table component of M for (c_out, c_in), and the force block it multiplies (3 = -X2)
__constant__ int c_ent[3][3] = {{0, 1, 4}, {1, 2, 5}, {4, 5, 3}};
__constant__ int c_bsel[3][3] = {{0, 1, 3}, {0, 1, 3}, {0, 1, 2}};

// Split x into NS pieces of the operand type; returned as raw bits (bf16 in
// the low 16 bits, or the tf32 bit pattern).  FP32 arithmetic throughout: each
// remainder x - bf16(x) is exact in FP32, and three bf16 pieces hold all 24
// bits of an FP32 value.
template <int PREC>
__device__ __forceinline__ void split(float x, uint32_t (&out)[TcCfg<PREC>::NS]) {
    if (PREC == FBC_PREC_TF32) {
        uint32_t t;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
        out[0] = t;
    } else {
        float r = x;
#pragma unroll
        for (int s = 0; s < TcCfg<PREC>::NS; s++) {
            const __nv_bfloat16 h = __float2bfloat16_rn(r);
            out[s] = (uint32_t)__bfloat16_as_ushort(h);
            r = __fsub_rn(r, __bfloat162float(h));
        }
    }
}

// 16 bytes of one core-matrix row: eight bf16 (low halves) or four tf32 words.
template <int ES, int KPC>
__device__ __forceinline__ uint4 pack16(const uint32_t (&w)[KPC]) {
    uint4 v;
    if (ES == 2) {
        v.x = w[0] | (w[1 % KPC] << 16);
        v.y = w[2 % KPC] | (w[3 % KPC] << 16);
        v.z = w[4 % KPC] | (w[5 % KPC] << 16);
        v.w = w[6 % KPC] | (w[7 % KPC] << 16);
    } else {
        v.x = w[0], v.y = w[1 % KPC], v.z = w[2 % KPC], v.w = w[3 % KPC];
    }
    return v;
}

template <int PREC>
__global__ void __launch_bounds__(kTileA, 1) k_contract_tc(ContractArgs A, int n_rhs, int* status) {
    using C = TcCfg<PREC>;
    constexpr int TA = kTileA, TB = kTileB;
    constexpr int KPC = 16 / C::ES;              // K elements per 16-byte core row
    constexpr int KCOL = C::KB / KPC;            // core matrices along K per block
    constexpr int SBO_A = KCOL * 128;            // bytes per 8-row group
    constexpr int ABLK = TA * C::KB * C::ES;     // bytes per A block
    constexpr int BBLK = kMaxNP * C::KB * C::ES; // bytes per B block (allocated for N = 128)
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase;
    __shared__ int s_abort;

    const int HW = A.H * A.W;
    unsigned char* sA = smem;                                  // [6][NS] blocks
    unsigned char* sB = sA + 6 * C::NS * ABLK;                  // [4][NS] blocks: X0, X1, X2, -X2
    float* s_tab = (float*)(sB + 4 * C::NS * BBLK);             // [6][HW]
    int* s_off = (int*)(s_tab + 6 * HW);                        // [TB]

    const int tA = blockIdx.x;
    const int k = A.k0 + blockIdx.y;
    const int r0 = blockIdx.z * kRhsPerCta;
    const int RG = min(kRhsPerCta, n_rhs - r0);
    const int NP = ((2 * RG + 15) / 16) * 16;
    const int a_loc = threadIdx.x;
    const int a = tA * TA + a_loc;
    const int2 xa = A.xy_p[a];
    const int4 bA = A.bbox_a[tA];
    const float* tk = A.tab32 + (size_t)(k - A.kbase) * A.Dy * A.Dx * 6;

    if (threadIdx.x == 0) {
        s_abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    const uint32_t id = idesc(C::FMT, TA, NP);
    uint32_t phase = 0;
    bool acc[3] = {false, false, false};
    bool pending = false;  // MMAs committed but not yet waited for

    for (int tB = 0; tB < A.n_tb && !s_abort; tB++) {
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
        for (int e = threadIdx.x; e < TB; e += TA) s_off[e] = A.off_i[tB * TB + e];
        __syncthreads();
        const int base = (xa.x - ox) + A.W * (xa.y - oy);
        for (int j0 = 0; j0 < TB; j0 += C::KB) {
            // the previous step's MMAs read the operand blocks: wait before overwriting them
            if (pending) {
                if (mbar_wait(&mbar, phase)) {
                    phase ^= 1u;
                    pending = false;
                } else if (threadIdx.x == 0) {
                    atomicExch(status, FBC_ERR_TIMEOUT);
                    s_abort = 1;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            __syncthreads();
            if (s_abort) break;
            // A blocks: row a_loc, columns j0 .. j0 + KB - 1, one table component at a time
#pragma unroll 1
            for (int kc = 0; kc < KCOL; kc++) {
                int idx[KPC];
#pragma unroll
                for (int i = 0; i < KPC; i++) idx[i] = base - s_off[j0 + kc * KPC + i];
                const uint32_t off = (a_loc / 8) * SBO_A + kc * 128 + (a_loc % 8) * 16;
#pragma unroll 1
                for (int eidx = 0; eidx < 6; eidx++) {
                    uint32_t pk[C::NS][KPC];
#pragma unroll
                    for (int i = 0; i < KPC; i++) {
                        uint32_t sp[C::NS];
                        split<PREC>(s_tab[eidx * HW + idx[i]], sp);
#pragma unroll
                        for (int s2 = 0; s2 < C::NS; s2++) pk[s2][i] = sp[s2];
                    }
#pragma unroll
                    for (int s2 = 0; s2 < C::NS; s2++)
                        *(uint4*)(sA + (eidx * C::NS + s2) * ABLK + off) = pack16<C::ES, KPC>(pk[s2]);
                }
            }
            // B blocks: rows n = 2 r + h (h = 0: x, 1: y'), columns j0 .. j0 + KB - 1; block 3 = -X2
            for (int p = threadIdx.x; p < NP * KCOL; p += TA) {
                const int n = p / KCOL, kc = p % KCOL;
                const int r = n >> 1, h = n & 1;
                const uint32_t off = (n / 8) * SBO_A + kc * 128 + (n % 8) * 16;
                const double* src = A.fh + (((size_t)(r0 + min(r, RG - 1)) * A.K + k) * A.NIpad +
                                            (size_t)tB * TB + j0 + kc * KPC) * 6 + h * 3;
#pragma unroll 1
                for (int c = 0; c < 4; c++) {
                    uint32_t pk[C::NS][KPC];
#pragma unroll
                    for (int i = 0; i < KPC; i++) {
                        float v = (r < RG) ? (float)src[i * 6 + (c < 3 ? c : 2)] : 0.0f;
                        if (c == 3) v = -v;
                        uint32_t sp[C::NS];
                        split<PREC>(v, sp);
#pragma unroll
                        for (int s2 = 0; s2 < C::NS; s2++) pk[s2][i] = sp[s2];
                    }
#pragma unroll
                    for (int s2 = 0; s2 < C::NS; s2++)
                        *(uint4*)(sB + (c * C::NS + s2) * BBLK + off) = pack16<C::ES, KPC>(pk[s2]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
                for (int co = 0; co < 3; co++) {
#pragma unroll 1
                    for (int ci = 0; ci < 3; ci++)
#pragma unroll 1
                        for (int pr = 0; pr < C::NPROD; pr++)
#pragma unroll 1
                            for (int s = 0; s < C::KB / C::KMMA; s++) {
                                const uint32_t aa = smem_u32(sA) + (c_ent[co][ci] * C::NS + c_prod_a[pr]) * ABLK + 256 * s;
                                const uint32_t bb = smem_u32(sB) + (c_bsel[co][ci] * C::NS + c_prod_b[pr]) * BBLK + 256 * s;
                                const uint64_t da = sdesc(aa, 128, SBO_A), db = sdesc(bb, 128, SBO_A);
                                const uint32_t accum = acc[co] ? 1u : 0u;
                                const uint32_t dt = tmem + (uint32_t)(co * NP);
                                if (C::FMT == 2)
                                    asm volatile(
                                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                                        "l"(da), "l"(db), "r"(id), "r"(accum));
                                else
                                    asm volatile(
                                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                                        "l"(da), "l"(db), "r"(id), "r"(accum));
                                acc[co] = true;
                            }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar)));
            }
            pending = true;
        }
    }
    // drain the last commit (bounded; after a timeout this is the second, last
    // bounded wait for our own tensor-core work), then read the accumulators
    bool ok = true;
    if (pending) {
        ok = mbar_wait(&mbar, phase);
        if (!ok && threadIdx.x == 0) atomicExch(status, FBC_ERR_TIMEOUT);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (ok && !s_abort) {
        const int warp = threadIdx.x / 32;
        for (int co = 0; co < 3; co++)
            for (int c0 = 0; c0 < NP; c0 += 16) {
                uint32_t v[16];
                const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(co * NP + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const int n = c0 + i, r = n >> 1, h = n & 1;
                    if (r < RG) {
                        double* o = A.uh + (((size_t)(r0 + r) * A.K + k) * A.NPpad + a) * 6 + h * 3 + co;
                        *o = (double)__uint_as_float(v[i]);
                    }
                }
            }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

template <int PREC>
size_t tc_smem(int HW) {
    using C = TcCfg<PREC>;
    return (size_t)6 * C::NS * kTileA * C::KB * C::ES + (size_t)4 * C::NS * kMaxNP * C::KB * C::ES +
           (size_t)6 * HW * 4 + (size_t)kTileB * 4 + 1024;
}

template <int PREC>
cudaError_t launch_tc(const ContractArgs& A, const Plan& P, int n_rhs, cudaStream_t st, int n_modes) {
    const size_t smem = tc_smem<PREC>(P.H * P.W);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_contract_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    dim3 grid(P.n_ta, n_modes, (n_rhs + kRhsPerCta - 1) / kRhsPerCta);
    k_contract_tc<PREC><<<grid, kTileA, smem, st>>>(A, n_rhs, P.d_status);
    return cudaGetLastError();
}

}  // namespace

size_t contract_tc_smem(int precision, int HW) {
    if (precision == FBC_PREC_TF32) return tc_smem<FBC_PREC_TF32>(HW);
    if (precision == FBC_PREC_BF16X2) return tc_smem<FBC_PREC_BF16X2>(HW);
    return tc_smem<FBC_PREC_BF16X3>(HW);
}

// Modes A.k0 .. A.k0 + n_modes - 1 (default: through K - 1) on the tensor cores (A.k0 >= 1).
cudaError_t launch_contract_tc(const ContractArgs& A, const Plan& P, int n_rhs, cudaStream_t st, int n_modes) {
    if (n_modes < 0) n_modes = P.K - A.k0;
    if (P.precision == FBC_PREC_TF32) return launch_tc<FBC_PREC_TF32>(A, P, n_rhs, st, n_modes);
    if (P.precision == FBC_PREC_BF16X2) return launch_tc<FBC_PREC_BF16X2>(A, P, n_rhs, st, n_modes);
    if (P.precision == FBC_PREC_BF16X3) return launch_tc<FBC_PREC_BF16X3>(A, P, n_rhs, st, n_modes);
    return cudaErrorInvalidValue;
}

}  // namespace fbc
