// FP64-accurate per-mode contraction on the tensor cores: fixed-point bf16
// slices with exact FP32 accumulation (Ozaki's error-free splitting of a dot
// product), for plans with several right-hand sides.
//
// The operation is the one of the other forms (Sec. 3.2, Eqs. 37-38 in the mode
// domain): for every mode k >= 1, pad column a and output component co,
//     U_co(a, n) = sum_{ci, b} M_{co ci}(x_a - x_b) X_ci(b, n),
// n over the x and y' halves of the right-hand sides.  Exactness comes from
// three facts:
//   * every operand value v is scaled by a power of two to |v'| < 1/2 and cut
//     into six slices t_1 .. t_6, t_i an integer of at most 8 bits times
//     2^(-8 i) (round to nearest, so the slices after the first are at most 128
//     units); six slices hold v' to 2^-49;
//   * the product of two slices is exact in FP32 (16 significant bits), and all
//     products t_i s_j with the same i + j = q lie on the grid 2^(-8 q);
//   * an FP32 accumulator that only ever adds values of one grid is exact while
//     the sum stays below 2^24 grid units.  With 192 terms per group (64
//     interface columns x 3 components) and at most q - 1 products of at most
//     2^14 units per term, the diagonals q = 2 .. 5 stay exact in the worst case.
// The 26 slice products with i, j <= 6 and i + j <= 8 are kept.  Diagonals 2, 3,
// 4 and 5 have an accumulator each in tensor memory; 6, 7 and 8 (about 2^-31 of
// the result) share a fifth, whose rounding stays near 2^-54 of the result.  The
// group's five sums are combined in double-float arithmetic, scaled back and
// added to a running double-float sum per output.  What is left out -- slices
// beyond the sixth and products with i + j > 8 -- is about 2^-47 of the largest
// operand product, per term.
//
// Scales: all table entries of a (pad tile, interface tile) pair share 2^E, the
// smallest power of two above twice their largest magnitude over the pair's
// 128 x 64 entries (of the CTA's three reals), so every cell of the pair's table
// sub-box is cut into slices once; the force column n of mode k shares 2^F(k, n),
// found by a reduction before the split.  Row and column scales factor out of the
// GEMM exactly.
//
// A CTA owns 128 pad columns (the GEMM rows, one tensor-memory lane each), one
// output component co, one mode and 32 right-hand sides (N = 64), and walks the
// interface columns tile by tile (64 columns, one accumulation group), in stages
// of 16:
//   * per tile, the eight builder warps stage the CTA's three reals of the
//     double-float sub-box (prefetched during the previous tile), find the
//     pair's scale and cut each cell into 18 bf16 slices in shared memory;
//   * per stage, they gather the slices of the co-th row of M, (M_{co 0},
//     M_{co 1}, M_{co 2}), and store them into tensor memory one input component
//     at a time (3 x 6 blocks of 128 x 16 bf16), each handed over by its own
//     barrier pair, so the stores of one component overlap the products of the
//     others;
//   * one thread streams the force operand, split once per apply (3 x 6 blocks
//     of 64 x 16 bf16 per stage, 36 KB), with bulk copies into a ring of stages;
//   * one thread issues 3 x 26 tcgen05.mma (M = 128, N = 64, K = 16) per stage
//     into the five accumulators;
//   * at the start of every tile the builders drain the previous tile's group
//     into their running double-float sums.
// Tensor memory: 5 x 64 accumulator columns and 18 x 8 columns of A: 464 of 512.
// The mode k = 0 stays with the double-float kernel, as in the other tensor forms.
//
// Every wait is bounded as in the other tensor-core kernel: pipeline waits give
// up after the plan's wait limit or once another role gave up; the waits for a
// CTA's own bulk copies and products in flight keep the full bound; a stopped CTA
// records the status word, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "fbc_internal.cuh"
#include "fbc_tc.cuh"

namespace fbc {
namespace {

constexpr int kTmemCols = 512;
constexpr int kRows = kTileA;        // GEMM rows (pad columns) per CTA
constexpr int kRhs = 32;             // right-hand sides per CTA
constexpr int kN = 2 * kRhs;         // GEMM columns: (x, y') of each right-hand side
constexpr int kKC = 16;              // interface columns per stage (the bf16 MMA's K)
constexpr int kStages = kTileB / kKC;  // stages per interface tile = per accumulation group
constexpr int kNS = 6;               // slices per operand value
constexpr int kNQ = 5;               // accumulators: diagonals q = 2, 3, 4, 5 and q >= 6 together
constexpr int kNPair = 26;           // slice products with i, j <= 6 and i + j <= 8
constexpr int kBuilderWarps = 8;
constexpr int kBuilders = kBuilderWarps * 32;
constexpr int kMmaWarp = 8, kCopyWarp = 9;
constexpr int kThreads = 10 * 32;
constexpr int kS = 3;                // force-operand ring stages
constexpr uint32_t kAcol = kNQ * kN;                     // first TMEM column of the A blocks (after 5 x 64)
constexpr uint32_t kAcols = 3 * kNS * 8;                 // TMEM columns of the A blocks (18 blocks of 128 x 16 bf16)
static_assert(kAcol + kAcols <= kTmemCols, "tensor memory");
constexpr uint32_t kBBlk = (uint32_t)kN * kKC * 2;       // one (ci, slice) block of a force chunk: 2 KB
constexpr uint32_t kChunk = 3u * kNS * kBBlk;            // one stage of the force operand: 36 KB
constexpr uint32_t kSBO = (kKC / 8) * 128;               // 8-row group stride of a [rows][16] bf16 block
constexpr uint32_t kSleepNs = 200;  // suspend hint of the copy thread's waits and the MMA thread's force waits
constexpr int kEmin = -120, kEmax = 120;                 // clamp of the scale exponents (2^E a normal float)

// Entry of M(d) in row co, column ci, as (index into the six table reals, sign):
// M = [[A11, A12, -B13], [A12, A22, -B23], [B13, B23, A33]], reals (A11, A12, A22, A33, B13, B23).
__host__ __device__ constexpr int oz_real(int co, int ci) {
    return co == 0 ? (ci == 0 ? 0 : ci == 1 ? 1 : 4) : co == 1 ? (ci == 0 ? 1 : ci == 1 ? 2 : 5) : (ci == 0 ? 4 : ci == 1 ? 5 : 3);
}
__host__ __device__ constexpr bool oz_neg(int co, int ci) { return ci == 2 && co < 2; }

// Slice products by diagonal: pair p multiplies A slice oz_pi(p) with B slice oz_pj(p) (1-based) into
// diagonal q = oz_pi(p) + oz_pj(p), accumulator oz_acc(p) (q = 6, 7, 8 share the last); oz_first(p) marks
// the first product into its accumulator.
__host__ __device__ constexpr int oz_pi(int p) {
    constexpr int v[kNPair] = {1, 1, 2, 1, 2, 3, 1, 2, 3, 4, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 6, 2, 3, 4, 5, 6};
    return v[p];
}
__host__ __device__ constexpr int oz_pj(int p) {
    constexpr int v[kNPair] = {1, 2, 1, 3, 2, 1, 4, 3, 2, 1, 5, 4, 3, 2, 1, 6, 5, 4, 3, 2, 1, 6, 5, 4, 3, 2};
    return v[p];
}
__host__ __device__ constexpr int oz_acc(int p) { return (oz_pi(p) + oz_pj(p) < 6 ? oz_pi(p) + oz_pj(p) : 6) - 2; }
__host__ __device__ constexpr bool oz_first(int p) { return p == 0 || oz_acc(p) != oz_acc(p - 1); }
static_assert(oz_pi(kNPair - 1) + oz_pj(kNPair - 1) == 8 && oz_first(10) && !oz_first(15) && !oz_first(21) &&
                  oz_acc(kNPair - 1) == kNQ - 1,
              "pair table");

// Six fixed-point slices of v' = (hi + lo) s, |v'| < 1/2, s a power of two: t_i is v's remainder
// rounded to the grid 2^(-8 i) (add and subtract 1.5 x 2^(23 - 8 i)).  hi s - t_1 and the later
// remainders are exact; only lo s joins with a rounding, of at most 2^-49.
__device__ __forceinline__ void oz_split(float hi, float lo, float s, float (&t)[kNS]) {
    const float C1 = 49152.0f, C2 = 192.0f, C3 = 0.75f;
    const float C4 = 0.0029296875f, C5 = 1.1444091796875e-05f, C6 = 4.470348358154297e-08f;
    t[0] = __fsub_rn(__fmaf_rn(hi, s, C1), C1);
    float r = __fmaf_rn(hi, s, -t[0]);
    t[1] = __fsub_rn(__fadd_rn(r, C2), C2);
    r = __fsub_rn(r, t[1]);
    t[2] = __fsub_rn(__fadd_rn(r, C3), C3);
    r = __fsub_rn(r, t[2]);
    r = __fmaf_rn(lo, s, r);
    t[3] = __fsub_rn(__fadd_rn(r, C4), C4);
    r = __fsub_rn(r, t[3]);
    t[4] = __fsub_rn(__fadd_rn(r, C5), C5);
    r = __fsub_rn(r, t[4]);
    t[5] = __fsub_rn(__fadd_rn(r, C6), C6);
}

// 2^-E as a float and the exponent E of a magnitude bound m: the smallest power of two above 2 m
// (|v| <= m gives |v 2^-E| < 1/2), clamped to [kEmin, kEmax].
__device__ __forceinline__ int oz_exp_of(float m) {
    const int e = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;  // floor(log2 m) (m = 0: -127)
    return min(max(e + 2, kEmin), kEmax);
}
__device__ __forceinline__ float oz_pow2(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }


// ---- force operand: scales and slices (once per apply) ----------------------

// Scale exponent F(k, n) of every force column (right-hand side r, half h) of modes k0 .. k0 + n_modes - 1:
// one block per (mode, rhs), the largest |fh| of the half over the interface columns and its three
// components, compared as the integer bits of the magnitudes.  fexp[(r K + k) 2 + h].
__global__ void __launch_bounds__(256) k_oz_fscale(const double* __restrict__ fh, int K, int NIpad, int k0,
                                                   int* __restrict__ fexp) {
    const int k = k0 + (int)blockIdx.x, r = (int)blockIdx.y;
    const double* src = fh + ((size_t)r * K + k) * NIpad * 6;
    unsigned long long m0 = 0ull, m1 = 0ull;  // halves x (entries 0..2) and y' (3..5)
    for (int i = threadIdx.x; i < NIpad * 3; i += blockDim.x) {  // one double2 per step: entries 2j, 2j + 1
        const double2 v = ((const double2*)src)[i];
        const int j = i % 3;
        const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & 0x7fffffffffffffffull;
        const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & 0x7fffffffffffffffull;
        if (j == 0) m0 = max(m0, max(a, b));
        else if (j == 1) m0 = max(m0, a), m1 = max(m1, b);
        else m1 = max(m1, max(a, b));
    }
    const unsigned long long m[2] = {m0, m1};
    __shared__ unsigned long long s_m[2][8];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        unsigned long long v = m[h];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x % 32 == 0) s_m[h][threadIdx.x / 32] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int h = threadIdx.x;
        unsigned long long v = 0ull;
        for (int w = 0; w < (int)blockDim.x / 32; w++) v = max(v, s_m[h][w]);
        const int e = (int)((v >> 52) & 0x7ffull) - 1023;  // floor(log2 max) (max = 0: -1023)
        fexp[((size_t)r * K + k) * 2 + h] = min(max(e + 2, kEmin), kEmax);
    }
}

// Chunk of the sliced force operand for (k, rhs group g, interface tile tB, stage st).
__host__ __device__ __forceinline__ size_t oz_chunk(int k, int g, int tB, int st, int G, int n_tb) {
    return (((size_t)k * G + g) * n_tb + tB) * kStages + st;
}

// One thread per (mode, rhs group g < Gu, tile, stage, rhs r of the group, core column kc): the eight interface
// columns b0 .. b0 + 7 of both halves and all three components of right-hand side r, each cut into six
// slices at its column's scale, stored as 16-byte core rows of the K-major blocks (ci, slice) of the
// chunk, GEMM column n = 2 r + h.  Right-hand sides at or beyond n_rhs are zero.
__global__ void __launch_bounds__(256) k_oz_prep(const double* __restrict__ fh, const int* __restrict__ fexp, int K,
                                                 int NIpad, int n_tb, int G, int Gu, int n_rhs, int k0, int n_modes,
                                                 unsigned char* __restrict__ out) {
    const size_t total = (size_t)n_modes * Gu * n_tb * kStages * kRhs * 2;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int kc = (int)(t & 1), rl = (int)((t >> 1) % kRhs);
        size_t q = t / (2 * kRhs);
        const int st = (int)(q % kStages);
        q /= kStages;
        const int tB = (int)(q % n_tb);
        q /= n_tb;
        const int g = (int)(q % Gu);
        const int k = k0 + (int)(q / Gu);
        const int r = g * kRhs + rl;
        const int b0 = tB * kTileB + st * kKC + kc * 8;
        unsigned char* chunk = out + oz_chunk(k, g, tB, st, G, n_tb) * kChunk;
        const double* src = fh + (((size_t)r * K + k) * NIpad + b0) * 6;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int n = 2 * rl + h;
            const float s = r < n_rhs ? oz_pow2(-fexp[((size_t)r * K + k) * 2 + h]) : 0.0f;
            const uint32_t off = (uint32_t)(n / 8) * kSBO + (uint32_t)kc * 128u + (uint32_t)(n % 8) * 16u;
#pragma unroll
            for (int ci = 0; ci < 3; ci++) {
                uint32_t w[kNS][4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    float t2[2][kNS];
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        const double x = r < n_rhs ? src[(size_t)(2 * i + u) * 6 + 3 * h + ci] : 0.0;
                        const float hi = d2f_int(x);
                        const float lo = d2f_int(x - f2d_int(hi));
                        oz_split(hi, lo, s, t2[u]);
                    }
#pragma unroll
                    for (int p = 0; p < kNS; p++)
                        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w[p][i]) : "f"(t2[1][p]), "f"(t2[0][p]));
                }
#pragma unroll
                for (int p = 0; p < kNS; p++)
                    *(uint4*)(chunk + (size_t)(ci * kNS + p) * kBBlk + off) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
            }
        }
    }
}

// ---- the contraction --------------------------------------------------------

struct OzArgs {
    ContractArgs A;              // table (double-float), uh, geometry; A.k0 = first mode of the launch
    const unsigned char* bprep;  // sliced force operand, chunks oz_chunk(k, g, tB, st)
    const int* fexp;             // force column scale exponents [rhs][K][2]
    int n_rhs, G;                // rhs applied, rhs groups of the buffer's layout
};

struct OzSync {
    uint64_t bfull[kS], empty[kS], done, afull[3], aempty[3];  // A: one barrier pair per input component
    uint32_t tbase;
    volatile int abort;
};

// Packed FP32 pairs (two lanes per instruction, each rounded to nearest as the scalar operation).
__device__ __forceinline__ uint64_t pk2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t r, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// oz_split on two values at once: (hi, lo) pairs of two values, s a pair of powers of two.
__device__ __forceinline__ void oz_split2(uint64_t hi, uint64_t lo, uint64_t s, uint64_t (&t)[kNS]) {
    const uint64_t C1 = pk2(49152.0f, 49152.0f), C2 = pk2(192.0f, 192.0f), C3 = pk2(0.75f, 0.75f);
    const uint64_t C4 = pk2(0.0029296875f, 0.0029296875f), C5 = pk2(1.1444091796875e-05f, 1.1444091796875e-05f);
    const uint64_t C6 = pk2(4.470348358154297e-08f, 4.470348358154297e-08f);
    const uint64_t m = mul2(hi, s);  // exact: s is a power of two
    t[0] = sub2(add2(m, C1), C1);
    uint64_t r = sub2(m, t[0]);
    t[1] = sub2(add2(r, C2), C2);
    r = sub2(r, t[1]);
    t[2] = sub2(add2(r, C3), C3);
    r = sub2(r, t[2]);
    r = fma2(lo, s, r);
    t[3] = sub2(add2(r, C4), C4);
    r = sub2(r, t[3]);
    t[4] = sub2(add2(r, C5), C5);
    r = sub2(r, t[4]);
    t[5] = sub2(add2(r, C6), C6);
}

__device__ __forceinline__ uint32_t cvt_bf16x2(float hi, float lo) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Two-sum (Knuth) on pairs: s + e == a + b exactly, per lane.
__device__ __forceinline__ void two_sum2(uint64_t a, uint64_t b, uint64_t& s, uint64_t& e) {
    s = add2(a, b);
    const uint64_t bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// Running double-float sums of two outputs: (H, L) += the five accumulator sums d[0..4] of a group (pairs:
// diagonals 2, 3, 4, 5 and 6-8), at the group's scale sc.  d2 + d3 + d4 by two-sums (they differ by about
// 2^8 each and are exact); the rest, below 2^-23 of the total, joins the low word.
__device__ __forceinline__ void oz_accumulate2(const uint64_t (&d)[kNQ], uint64_t sc, uint64_t& H, uint64_t& L) {
    uint64_t s, e, s2, e2, t;
    two_sum2(d[0], d[1], s, e);
    two_sum2(s, d[2], s2, e2);
    uint64_t l = add2(add2(add2(e, e2), d[3]), d[4]);
    s2 = mul2(s2, sc);
    l = mul2(l, sc);
    two_sum2(H, s2, H, t);
    L = add2(L, add2(t, l));
}

// Shared-memory bytes of one staged table sub-box: the CTA's three reals as (hi, lo) of the first two
// (packed pairs), hi and lo of the third, and the largest |hi| of the three per entry.
__host__ __device__ inline size_t oz_tab_bytes(int HW) { return ((size_t)HW * 28 + 15) / 16 * 16; }

__global__ void __launch_bounds__(kThreads, 1) k_contract_oz(OzArgs O, int wl, int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ OzSync sy;
    const ContractArgs& A = O.A;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int co = (int)blockIdx.x % 3, tA = (int)blockIdx.x / 3;
    const int k = A.k0 + (int)blockIdx.y, g = (int)blockIdx.z;
    const int n_it = A.n_tb * kStages;
    const int HW = A.H * A.W;
    const size_t tb = oz_tab_bytes(HW);
    unsigned char* sB = smem;                                     // [kS][kChunk]
    unsigned char* s_tabs = smem + kS * kChunk;                   // [tb]: the staged double-float sub-box
    int* s_off = (int*)(s_tabs + tb);                             // [2][kTileB]: interface offsets of two tiles
    uint32_t* s_sl = (uint32_t*)(s_off + 2 * kTileB);             // [HW][9]: the sub-box cut into slices
    __shared__ uint32_t s_wmax[kBuilderWarps];
    volatile int& s_abort = sy.abort;

    if (threadIdx.x == 0) {
        sy.abort = 0;
        for (int s = 0; s < kS; s++) tc::mbar_init(&sy.bfull[s], 1), tc::mbar_init(&sy.empty[s], 1);
        tc::mbar_init(&sy.done, 1);
        for (int c = 0; c < 3; c++) tc::mbar_init(&sy.afull[c], kBuilderWarps), tc::mbar_init(&sy.aempty[c], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&sy.tbase)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sy.tbase;

    if (warp == kCopyWarp) {
        // ---- force operand: one bulk copy per stage ----
        if (lane == 0) {
            int il = 0;
            for (; il < n_it; il++) {
                const int s = il % kS;
                const uint32_t u = (uint32_t)(il / kS);
                if (!tc::wait_or_abort_sleep(&sy.empty[s], (u & 1u) ^ 1u, &s_abort, wl, kSleepNs)) {
                    s_abort = 1;
                    break;
                }
                const int tB = il / kStages, st = il % kStages;
                tc::mbar_expect_tx(&sy.bfull[s], kChunk);
                tc::bulk_g2s(sB + (size_t)s * kChunk, O.bprep + oz_chunk(k, g, tB, st, O.G, A.n_tb) * kChunk, kChunk,
                             &sy.bfull[s]);
            }
            // copies still in flight land before the CTA may go on or exit: the full bound, whatever the stop flag
            for (int j = max(0, il - kS); j < il; j++) tc::mbar_wait(&sy.bfull[j % kS], (uint32_t)(j / kS) & 1u);
        }
    } else if (warp == kMmaWarp) {
        // ---- tensor-core issue: 3 x 26 products per stage ----
        if (lane == 0) {
            const uint32_t id = tc::idesc(1, kRows, kN);
            const uint64_t dB0 = tc::sdesc(tc::smem_u32(sB), 128, kSBO);
            for (int il = 0; il < n_it; il++) {
                const int s = il % kS;
                const uint32_t par = (uint32_t)(il / kS) & 1u;
                if (!tc::wait_or_abort_sleep(&sy.bfull[s], par, &s_abort, wl, kSleepNs)) {
                    s_abort = 1;
                    break;
                }
                const uint64_t dBs = dB0 + (uint64_t)(((size_t)s * kChunk) >> 4);
                const uint32_t ta0 = tmem + kAcol;
                const bool first = (il % kStages) == 0;  // a new group overwrites the accumulators
                bool stop = false;
#pragma unroll
                for (int ci = 0; ci < 3; ci++) {
                    // the A blocks of input component ci, stored by the builders while the others' products run
                    if (!tc::wait_or_abort(&sy.afull[ci], (uint32_t)il & 1u, &s_abort, wl)) {
                        stop = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                    for (int p = 0; p < kNPair; p++) {
                        const uint32_t ta = ta0 + (uint32_t)(ci * kNS + oz_pi(p) - 1) * 8u;
                        const uint64_t db = dBs + (uint64_t)(((uint32_t)(ci * kNS + oz_pj(p) - 1) * kBBlk) >> 4);
                        const uint32_t dt = tmem + (uint32_t)oz_acc(p) * (uint32_t)kN;
                        const uint32_t en = (first && ci == 0 && oz_first(p)) ? 0u : 1u;
                        asm volatile(
                            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dt),
                            "r"(ta), "l"(db), "r"(id), "r"(en));
                    }
                    tc::commit(&sy.aempty[ci]);
                }
                if (stop) {
                    s_abort = 1;
                    break;
                }
                tc::commit(&sy.empty[s]);
            }
            tc::commit(&sy.done);  // also after a stop: fires once the issued products are complete
        }
    } else {
        // ---- builders (warps 0..7): table slices into tensor memory, drains, output ----
        const int tid = threadIdx.x;               // 0 .. 255
        const int a_loc = (warp & 3) * 32 + lane;  // TMEM lane = GEMM row
        const int hb = warp >> 2;                  // which 8 of a stage's 16 columns, which 16 of the 32 GEMM columns
        const int a = tA * kRows + a_loc;
        const int2 xa = A.xy_p[a];
        const int4 bA = A.bbox_a[tA];
        const float* tk = A.tabx2 + (size_t)k * A.Dy * A.Dx * 12;
        const int rl0 = oz_real(co, 0), rl1 = oz_real(co, 1), rl2 = oz_real(co, 2);
        const float sg2 = oz_neg(co, 2) ? -1.0f : 1.0f;
        // the CTA's three reals of every entry of tile tB's sub-box into the staging buffer (hi/lo pairs of
        // the first two, hi and lo of the third), and the tile's interface offsets into offset buffer tB & 1,
        // by asynchronous 4-byte copies
        auto stage_async = [&](int tB) {
            const int4 bB = A.bbox_b[tB];
            const int ox = bA.x - bB.y, oy = bA.z - bB.w;
            float* h01 = (float*)s_tabs;
            float* l01 = h01 + 2 * HW;
            float* h2 = l01 + 2 * HW;
            float* l2 = h2 + HW;
            for (int e = tid; e < HW; e += kBuilders) {
                const int iy = e / A.W, ix = e - iy * A.W;
                const int gx = ox + ix - A.box_x0, gy = oy + iy - A.box_y0;
                const bool in = gx < A.Dx && gy < A.Dy;
                const float* src = in ? tk + ((size_t)gy * A.Dx + gx) * 12 : tk;  // zero outside the box
                const int nb = in ? 4 : 0;
                tc::cp_async4(h01 + 2 * e, src + 2 * rl0, nb);
                tc::cp_async4(h01 + 2 * e + 1, src + 2 * rl1, nb);
                tc::cp_async4(l01 + 2 * e, src + 2 * rl0 + 1, nb);
                tc::cp_async4(l01 + 2 * e + 1, src + 2 * rl1 + 1, nb);
                tc::cp_async4(h2 + e, src + 2 * rl2, nb);
                tc::cp_async4(l2 + e, src + 2 * rl2 + 1, nb);
            }
            if (tid < kTileB / 4) tc::cp_async16(s_off + (tB & 1) * kTileB + 4 * tid, A.off_i + tB * kTileB + 4 * tid);
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        // running double-float sums of this thread's row and GEMM columns hb * 32 .. + 31, as pairs of columns
        uint64_t H[16], L[16];
#pragma unroll
        for (int j = 0; j < 16; j++) H[j] = 0ull, L[j] = 0ull;
        const uint32_t tacc = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(hb * 32);
        auto drain = [&](float sc) {
            const uint64_t sc2 = pk2(sc, sc);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                uint32_t u[kNQ][8];
#pragma unroll
                for (int q = 0; q < kNQ; q++) tc::ld8_nowait(tacc + (uint32_t)(q * kN + c * 8), u[q]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    uint64_t d[kNQ];
#pragma unroll
                    for (int q = 0; q < kNQ; q++) d[q] = pk2(__uint_as_float(u[q][2 * j]), __uint_as_float(u[q][2 * j + 1]));
                    oz_accumulate2(d, sc2, H[c * 4 + j], L[c * 4 + j]);
                }
            }
        };
        const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + kAcol + 4u * (uint32_t)hb;
        float sc_prev = 0.0f;  // 2^E of the tile whose group is drained next
        int il = 0;
        stage_async(0);
        for (int tB = 0; tB < A.n_tb; tB++) {
            asm volatile("cp.async.wait_all;" ::: "memory");
            // this tile's copies are visible to every builder, and every builder is done with the previous
            // tile's slices; one stop decision
            if (tc::builders_sync_any(s_abort)) break;
            const uint64_t* h01 = (const uint64_t*)s_tabs;
            const uint64_t* l01 = h01 + HW;
            const float* h2 = (const float*)(l01 + HW);
            const float* l2 = h2 + HW;
            float* me = (float*)(l2 + HW);
            for (int e = tid; e < HW; e += kBuilders) {
                float x0, x1;
                upk2(h01[e], x0, x1);
                me[e] = fmaxf(fabsf(h2[e]), fmaxf(fabsf(x0), fabsf(x1)));
            }
            if (tc::builders_sync_any(s_abort)) break;
            const int* off_b = s_off + (tB & 1) * kTileB;
            const int4 bB = A.bbox_b[tB];
            const int ox = bA.x - bB.y, oy = bA.z - bB.w;
            const int base = (xa.x - ox) + A.W * (xa.y - oy);
            // the tile pair's scale: the largest entry over its 128 x 64 pairs (each thread: its row and half
            // the columns; magnitudes compare as integers)
            float m = 0.0f;
#pragma unroll 8
            for (int j = hb * 32; j < hb * 32 + 32; j++) m = fmaxf(m, me[base - off_b[j]]);
            const uint32_t mw = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
            if (lane == 0) s_wmax[warp] = mw;
            if (tc::builders_sync_any(s_abort)) break;
            uint32_t mb = s_wmax[0];
#pragma unroll
            for (int w8 = 1; w8 < kBuilderWarps; w8++) mb = max(mb, s_wmax[w8]);
            const int E = oz_exp_of(__uint_as_float(mb));
            const float s_in = oz_pow2(-E), sc = oz_pow2(E);
            const uint64_t s01 = pk2(s_in, s_in), s22 = pk2(sg2 * s_in, sg2 * s_in);
            // every cell of the sub-box cut once at that scale: 18 bf16 slices (real, slice) in 9 words; cells
            // e0 and e0 + 256 go together (the third real split as a pair of cells; past the end, the last
            // cell again, written twice with the same bits)
            for (int e0 = tid; e0 < HW; e0 += 2 * kBuilders) {
                const int e1 = min(e0 + kBuilders, HW - 1);
                uint64_t t0[kNS], t1[kNS], t2[kNS];
                oz_split2(h01[e0], l01[e0], s01, t0);
                oz_split2(h01[e1], l01[e1], s01, t1);
                oz_split2(pk2(h2[e0], h2[e1]), pk2(l2[e0], l2[e1]), s22, t2);
                uint32_t* c0 = s_sl + 9 * e0;
                uint32_t* c1 = s_sl + 9 * e1;
#pragma unroll
                for (int q = 0; q < 3; q++) {  // word q of a real: slices 2q (low half) and 2q + 1
                    float a0, b0, a1, b1, x0, x1, y0, y1;
                    upk2(t0[2 * q], a0, b0);
                    upk2(t0[2 * q + 1], a1, b1);
                    c0[q] = cvt_bf16x2(a1, a0), c0[3 + q] = cvt_bf16x2(b1, b0);
                    upk2(t1[2 * q], a0, b0);
                    upk2(t1[2 * q + 1], a1, b1);
                    c1[q] = cvt_bf16x2(a1, a0), c1[3 + q] = cvt_bf16x2(b1, b0);
                    upk2(t2[2 * q], x0, x1);
                    upk2(t2[2 * q + 1], y0, y1);
                    c0[6 + q] = cvt_bf16x2(y0, x0), c1[6 + q] = cvt_bf16x2(y1, x1);
                }
            }
            if (tc::builders_sync_any(s_abort)) break;
            // the staging buffer is free: the next tile's sub-box loads while this tile's stages run
            if (tB + 1 < A.n_tb) stage_async(tB + 1);
            for (int st = 0; st < kStages; st++, il++) {
                const uint32_t ph = ((uint32_t)il & 1u) ^ 1u;  // parity of stage il - 1's phase
                int cell[8];  // row a_loc, interface columns st * 16 + hb * 8 .. + 7
#pragma unroll
                for (int i = 0; i < 8; i++) cell[i] = 9 * (base - off_b[st * kKC + hb * 8 + i]);
#pragma unroll
                for (int ci = 0; ci < 3; ci++) {
                    // the six slices of component ci, two columns per 32-bit word (words 3 ci .. 3 ci + 2 of
                    // a cell hold its slices 0 .. 5)
                    uint32_t w[kNS][4];
#pragma unroll
                    for (int i2 = 0; i2 < 4; i2++)
#pragma unroll
                        for (int q = 0; q < 3; q++) {
                            const uint32_t u0 = s_sl[cell[2 * i2] + 3 * ci + q], u1 = s_sl[cell[2 * i2 + 1] + 3 * ci + q];
                            w[2 * q][i2] = __byte_perm(u0, u1, 0x5410);
                            w[2 * q + 1][i2] = __byte_perm(u0, u1, 0x7632);
                        }
                    // component ci's blocks are free once stage il - 1's products of ci are complete; at a
                    // tile's first stage the whole of stage il - 1 (its last component) first, since the
                    // previous tile's group is drained before these stores.  The warp decides as one (the
                    // stores are warp-wide).
                    const bool tile_start = ci == 0 && st == 0 && tB > 0;
                    bool ok = !s_abort && tc::wait_or_abort(&sy.aempty[tile_start ? 2 : ci], ph, &s_abort, wl);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) {
                        s_abort = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    if (tile_start) drain(sc_prev);
#pragma unroll
                    for (int p = 0; p < kNS; p++)
                        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                                         trow + (uint32_t)(ci * kNS + p) * 8u),
                                     "r"(w[p][0]), "r"(w[p][1]), "r"(w[p][2]), "r"(w[p][3])
                                     : "memory");
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&sy.afull[ci]);
                }
            }
            sc_prev = sc;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");  // a prefetch still in flight after a stop
        // every product the MMA thread issued is complete once `done` fires (it commits on every path), so
        // this wait keeps the full bound whatever the stop flag says
        const bool done_ok = tc::mbar_wait(&sy.done, 0u);
        const bool ok = __all_sync(0xffffffffu, done_ok && !s_abort);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok) {
            drain(sc_prev);  // the last tile's group
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const int n = hb * 32 + j, r = g * kRhs + n / 2, h = n & 1;
                if (r < O.n_rhs) {
                    float hv0, hv1, lv0, lv1;
                    upk2(H[j / 2], hv0, hv1);
                    upk2(L[j / 2], lv0, lv1);
                    const float hv = (j & 1) ? hv1 : hv0, lv = (j & 1) ? lv1 : lv0;
                    const float sF = oz_pow2(O.fexp[((size_t)r * A.K + k) * 2 + h]);
                    A.uh[(((size_t)r * A.K + k) * A.NPpad + a) * 6 + 3 * h + co] =
                        f2d_int(__fmul_rn(hv, sF)) + f2d_int(__fmul_rn(lv, sF));
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && sy.abort) atomicExch(status, FBC_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

size_t oz_smem(int HW) {
    return (size_t)kS * kChunk + oz_tab_bytes(HW) + 2 * kTileB * 4 + (size_t)HW * 36 + 1024;
}
int oz_groups(const Plan& P) { return (P.opt.max_rhs + kRhs - 1) / kRhs; }
size_t oz_chunk_bytes(const Plan& P) { return (size_t)P.K * oz_groups(P) * P.n_tb * kStages * kChunk; }

}  // namespace

size_t contract_oz_smem(int HW) { return oz_smem(HW); }
int contract_oz_rhs_group() { return kRhs; }

// the sliced force operand of every mode and rhs group, then the scale exponents [max_rhs][K][2]
size_t contract_oz_prep_bytes(const Plan& P) {
    return oz_chunk_bytes(P) + (size_t)P.opt.max_rhs * P.K * 2 * sizeof(int);
}

// Modes A.k0 .. K - 1 (A.k0 >= 1) of an FBC_PREC_BF16X6 plan: scales and slices of the forces, then the
// contraction, one CTA per (pad tile, output component) x mode x group of 16 right-hand sides.
cudaError_t launch_contract_oz(const ContractArgs& A, const Plan& P, int n_rhs, cudaStream_t st) {
    const int n_modes = P.K - A.k0;
    if (n_modes <= 0 || n_rhs < 1) return cudaSuccess;
    const int HW = P.H * P.W;
    const size_t smem = oz_smem(HW);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    if (!P.d_bprep || P.bprep_prec != FBC_PREC_BF16X6 || P.bprep_bytes < contract_oz_prep_bytes(P) ||
        n_rhs > P.opt.max_rhs || !A.tabx2 || A.tabx2 != P.d_table_x2)
        return cudaErrorInvalidValue;
    OzArgs O;
    O.A = A;
    O.bprep = (const unsigned char*)P.d_bprep;
    O.fexp = (const int*)((const unsigned char*)P.d_bprep + oz_chunk_bytes(P));
    O.n_rhs = n_rhs;
    O.G = oz_groups(P);
    k_oz_fscale<<<dim3(n_modes, n_rhs), 256, 0, st>>>(A.fh, P.K, P.NIpad, A.k0, (int*)O.fexp);
    if (cudaError_t e = cudaGetLastError()) return e;
    const int gu = (n_rhs + kRhs - 1) / kRhs;  // rhs groups of this apply
    const size_t total = (size_t)n_modes * gu * P.n_tb * kStages * kRhs * 2;
    const int grid = (int)std::min<size_t>((total + 255) / 256, (size_t)152 * 32);
    k_oz_prep<<<grid, 256, 0, st>>>(A.fh, O.fexp, P.K, P.NIpad, P.n_tb, O.G, gu, n_rhs, A.k0, n_modes,
                                    (unsigned char*)P.d_bprep);
    if (cudaError_t e = cudaGetLastError()) return e;
    cudaError_t e = cudaFuncSetAttribute(k_contract_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    const int wl = P.wait_limit > 0 ? P.wait_limit : tc::kWaitLimit;
    k_contract_oz<<<dim3(3 * P.n_ta, n_modes, gu), kThreads, smem, st>>>(O, wl, P.d_status);
    return cudaGetLastError();
}

}  // namespace fbc
