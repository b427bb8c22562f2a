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
// right-hand sides (N = 2 R columns) and walks the interface columns in
// stages of 16, through a ring of shared-memory stages:
//   * eight builder warps gather the six 128 x 16 blocks A_e(a, b) =
//     T_e(x_a - x_b) from the staged table sub-box, split them into bf16
//     pieces (h, m, l) or round them to tf32, and store them in the K-major
//     no-swizzle canonical layout (8-row x 16-byte core matrices);
//   * the force operand X_0, X_1, X_2 was split once per apply by k_prep_b
//     into the same layout, one contiguous chunk per (k, rhs group, stage);
//     one thread streams each chunk in with a bulk copy (cp.async.bulk);
//   * one thread issues the 9 block products per split-product pair with
//     tcgen05.mma (M = 128, N = 2 R, K = 16 bf16 / 8 tf32) into three TMEM
//     accumulators (one per output component); the -B13, -B23 entries use
//     the instruction's negate-A bit; a commit to the stage's "empty" barrier
//     hands the stage back to the builders and the copy thread.
// Split products: TF32 (1), BF16X2 (hh + hm + mh), BF16X3 (+ hl + lh + mm),
// pieces h = bf16(x), m = bf16(x - h), l = bf16(x - h - m), all rounded to
// nearest.  The logarithmic k = 0 mode is left to the double-float kernel.
//
// Every wait is bounded.  The pipeline waits (stage hand-offs between the
// roles) give up after the plan's wait limit, or at once when another role has
// given up; on a timeout the CTA records the status word, stops, waits for its
// own bulk copies and tensor-core work -- those two waits ignore the stop and
// keep the full bound, since the CTA may not exit or free its tensor memory
// while either is in flight -- frees its tensor memory and returns.  Warps that
// synchronise on a named barrier decide to stop only right after it, so none
// is left waiting there.
#include <cuda_bf16.h>

#include <algorithm>

#include "fbc_internal.cuh"
#include "fbc_tc.cuh"

namespace fbc {
namespace {

constexpr int kTmemCols = 512;
constexpr int kRows = kTileA;    // GEMM rows (pad columns) per CTA
constexpr int kRhsPerCta = 64;
constexpr int kNPB = 128;        // force-operand rows per CTA (64 rhs x (x, y'))
constexpr int kKC = 16;          // interface columns per stage
constexpr int kBuilderWarps = 8;
constexpr int kBuilders = kBuilderWarps * 32;
constexpr int kMmaWarp = 8, kCopyWarp = 9;
constexpr int kThreads = 10 * 32;
constexpr int kStagesPerTile = kTileB / kKC;
constexpr int kDrainTiles = 16;  // interface tiles per tensor-memory accumulation group
constexpr uint32_t kAcol = 384;  // first TMEM column of the A operand (after 3 x 128 accumulator columns)

using tc::idesc;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::sdesc;
using tc::smem_u32;

template <int PREC>
struct TcCfg;
template <>
struct TcCfg<FBC_PREC_TF32> {
    static constexpr int ES = 4, NS = 1, NPROD = 1, KMMA = 8, FMT = 2, S = 3;
    static constexpr bool ATM = true;  // A operand in tensor memory
};
template <>
struct TcCfg<FBC_PREC_BF16X2> {
    static constexpr int ES = 2, NS = 2, NPROD = 3, KMMA = 16, FMT = 1, S = 3;
    static constexpr bool ATM = true;
};
template <>
struct TcCfg<FBC_PREC_BF16X3> {
    static constexpr int ES = 2, NS = 3, NPROD = 6, KMMA = 16, FMT = 1, S = 1;
    static constexpr bool ATM = false;  // 18 A blocks do not fit beside the accumulators
};

template <int PREC>
struct TcLayout {
    using C = TcCfg<PREC>;
    static constexpr int KPC = 16 / C::ES;                    // K elements per 16-byte core row
    static constexpr uint32_t SBO = (kKC / KPC) * 128;        // bytes per 8-row group of a [rows][16] block
    static constexpr size_t ABLK = (size_t)kRows * kKC * C::ES;
    static constexpr size_t A_STAGE = C::ATM ? 0 : 6 * C::NS * ABLK;  // shared-memory A stage
    static constexpr uint32_t ACOLS = (uint32_t)(kKC * C::ES / 4);         // TMEM columns of one A block
    static constexpr size_t B_STAGE = 3 * C::NS * (size_t)kNPB * kKC * C::ES;  // allocated for 128 rows
};

// Products issued per stage, fully unrolled: for output component co and
// input component ci the table entry kEnt[co][ci] of M (the (0, 2) and (1, 2)
// entries negated through the instruction descriptor), and for split product
// pr the pieces (kPa[pr], kPb[pr]) of the A and B operands, by decreasing
// magnitude: hh, hm, mh, hl, lh, mm.

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

// 16 bytes of one core-matrix row from KPC elements
template <int ES, int KPC>
__device__ __forceinline__ uint4 pack16(const uint32_t* w) {
    uint4 v;
    if (ES == 2) {
        v.x = w[0] | (w[1] << 16), v.y = w[2] | (w[3] << 16);
        v.z = w[4] | (w[5] << 16), v.w = w[6] | (w[7] << 16);
    } else {
        v.x = w[0], v.y = w[1], v.z = w[2], v.w = w[3];
    }
    return v;
}

using tc::builders_sync_any;
using tc::bulk_g2s;
using tc::cp_async16;
using tc::cp_async8;
using tc::mbar_arrive;
using tc::wait_or_abort;

// Chunk of the split force operand for (k, rhs group g, interface tile tB, stage st).
__host__ __device__ __forceinline__ size_t bchunk_index(int k, int g, int tB, int st, int G, int n_tb) {
    return (((size_t)k * G + g) * n_tb + tB) * kStagesPerTile + st;
}

// One thread per 16-byte core row (block c, row n, core column kc) of a chunk:
// X_c(b, n = 2 r + h) = fh[g rpc + r][k][b][3 h + c], zero for r beyond the group
// (rpc right-hand sides per group, G groups, npb >= 2 rpc rows per chunk).
template <int PREC>
__global__ void k_prep_b(const double* __restrict__ fh, int K, int NIpad, int n_tb, int G, int npb, int rpc,
                         int n_rhs, int k0, int n_modes, unsigned char* __restrict__ out) {
    using C = TcCfg<PREC>;
    using Lt = TcLayout<PREC>;
    constexpr int KPC = Lt::KPC, NKC = kKC / KPC;
    const size_t chunk_bytes = (size_t)3 * C::NS * npb * kKC * C::ES;
    const size_t per_chunk = (size_t)3 * npb * NKC;
    const size_t total = (size_t)n_modes * G * n_tb * kStagesPerTile * per_chunk;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        size_t q = t / per_chunk;
        const int rem = (int)(t % per_chunk);
        const int c = rem / (npb * NKC), n = (rem / NKC) % npb, kc = rem % NKC;
        const int st = (int)(q % kStagesPerTile);
        q /= kStagesPerTile;
        const int tB = (int)(q % n_tb);
        q /= n_tb;
        const int g = (int)(q % G);
        const int k = k0 + (int)(q / G);
        const int RG = min(rpc, n_rhs - g * rpc);
        const int r = n >> 1, h = n & 1;
        const int b0 = tB * kTileB + st * kKC + kc * KPC;
        uint32_t w[C::NS][KPC];
#pragma unroll
        for (int i = 0; i < KPC; i++) {
            float v = 0.f;
            if (r < RG) v = (float)fh[(((size_t)(g * rpc + r) * K + k) * NIpad + b0 + i) * 6 + h * 3 + c];
            uint32_t sp[C::NS];
            split<PREC>(v, sp);
#pragma unroll
            for (int p = 0; p < C::NS; p++) w[p][i] = sp[p];
        }
        unsigned char* base = out + bchunk_index(k, g, tB, st, G, n_tb) * chunk_bytes;
        const uint32_t off = (uint32_t)(n / 8) * Lt::SBO + kc * 128 + (n % 8) * 16;
#pragma unroll
        for (int p = 0; p < C::NS; p++)
            *(uint4*)(base + (size_t)(c * C::NS + p) * npb * kKC * C::ES + off) = pack16<C::ES, KPC>(w[p]);
    }
}

// Shared-memory barriers and flags of the contraction CTA.
template <int S>
struct TcSync {
    uint64_t full[S], bfull[S], empty[S], done, afull, aempty;
    uint32_t tbase;
    volatile int abort;
};

// One work item (job J, mode k = wk.y, pad tile tA = wk.z, rhs group g = wk.w) on the whole CTA.  it_base:
// stages this CTA has run before the item (every role counts alike, so stage s = it % S and the barrier
// phases run on across items); n_done: items run before it (the parity of `done`).
template <int PREC>
__device__ __forceinline__ void tc_item(const TcJob& J, const int4 wk, const uint32_t it_base, const uint32_t n_done,
                                        TcSync<TcCfg<PREC>::S>& sy, unsigned char* smem, const int wl) {
    using C = TcCfg<PREC>;
    using Lt = TcLayout<PREC>;
    constexpr int S = C::S;
    uint64_t* full = sy.full;
    uint64_t* bfull = sy.bfull;
    uint64_t* empty = sy.empty;
    uint64_t& done = sy.done;
    uint64_t& afull = sy.afull;
    uint64_t& aempty = sy.aempty;
    volatile int& s_abort = sy.abort;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const ContractArgs& A = J.A;
    {
        const uint32_t tmem = sy.tbase;
        const int HW = A.H * A.W;
        unsigned char* sA = smem;                                   // [S][6][NS][128][16]
        unsigned char* sB = sA + S * Lt::A_STAGE;                   // [S][3][NS][npb][16]
        int* s_off = (int*)(sB + S * Lt::B_STAGE);                  // [nbuf][TB]
        float* s_tab = (float*)(s_off + J.nbuf * kTileB);           // [nbuf][HW][6]
        const int nbuf = J.nbuf, gs = J.gs;
        const int k = wk.y, tA = wk.z, g = wk.w;
        const int r0 = g * J.rpc;
        const int RG = min(J.rpc, J.n_rhs - r0);
        const int NP = ((2 * RG + 15) / 16) * 16;
        const int n_it = A.n_tb * kStagesPerTile;
        const uint32_t chunk_bytes = (uint32_t)(3 * C::NS * J.npb * kKC * C::ES);
        const size_t bblk = (size_t)J.npb * kKC * C::ES;              // one (block, piece) of a chunk

        if (warp == kCopyWarp) {
            // ---- force operand: one bulk copy per stage ----
            if (lane == 0) {
                int il = 0;
                for (; il < n_it; il++) {
                    const uint32_t it = it_base + il;
                    const int s = it % S;
                    const uint32_t u = it / S;
                    if (!wait_or_abort(&empty[s], (u & 1u) ^ 1u, &s_abort, wl)) {
                        s_abort = 1;
                        break;
                    }
                    const int tB = il / kStagesPerTile, st = il % kStagesPerTile;
                    mbar_expect_tx(&bfull[s], chunk_bytes);
                    bulk_g2s(sB + s * Lt::B_STAGE, J.bprep + bchunk_index(k, g, tB, st, J.G, A.n_tb) * chunk_bytes,
                             chunk_bytes, &bfull[s]);
                }
                // copies still in flight land before the CTA may go on or exit: the full bound, whatever the
                // stop flag says
                for (int j = max(0, il - S); j < il; j++) {
                    const uint32_t it = it_base + j;
                    tc::mbar_wait(&bfull[it % S], (it / S) & 1u);
                }
            }
        } else if (warp == kMmaWarp) {
            // ---- tensor-core issue ----
            if (lane == 0) {
                const uint32_t id = idesc(C::FMT, kRows, NP), idn = id | (1u << 13);  // bit 13: negate A
                // descriptor of B block 0 of stage 0; the others differ by (byte offset >> 4) in the address field
                const uint64_t dB0 = sdesc(smem_u32(sB), 128, Lt::SBO);
                const uint64_t dA0 = sdesc(smem_u32(sA), 128, Lt::SBO);
                const uint32_t bblk16 = (uint32_t)(bblk >> 4);
                int gpos = 0;  // position of the stage in its accumulation group
                for (int il = 0; il < n_it; il++) {
                    const uint32_t it = it_base + il;
                    const int s = it % S;
                    const uint32_t par = (it / S) & 1u;
                    uint64_t* af = C::ATM ? &afull : &full[s];
                    const uint32_t apar = C::ATM ? (it & 1u) : par;
                    if (!wait_or_abort(af, apar, &s_abort, wl) || !wait_or_abort(&bfull[s], par, &s_abort, wl)) {
                        s_abort = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t dBs = dB0 + (uint64_t)((s * Lt::B_STAGE) >> 4);
                    const uint64_t dAs = dA0 + (uint64_t)((s * Lt::A_STAGE) >> 4);
                    // a new accumulation group starts by overwriting the accumulators
                    const uint32_t first = gpos == 0 ? 0u : 1u;
                    if (++gpos == gs) gpos = 0;
#pragma unroll
                    for (int co = 0; co < 3; co++)
#pragma unroll
                        for (int ci = 0; ci < 3; ci++)
#pragma unroll
                            for (int pr = 0; pr < C::NPROD; pr++)
#pragma unroll
                                for (int ks = 0; ks < kKC / C::KMMA; ks++) {
                                    constexpr int kEnt[3][3] = {{0, 1, 4}, {1, 2, 5}, {4, 5, 3}};
                                    constexpr int kPa[6] = {0, 0, 1, 0, 2, 1}, kPb[6] = {0, 1, 0, 2, 0, 1};
                                    const int ablk = kEnt[co][ci] * C::NS + kPa[pr];
                                    const uint64_t db = dBs + (uint64_t)((ci * C::NS + kPb[pr]) * bblk16 + 16 * ks);
                                    const uint32_t idd = (ci == 2 && co < 2) ? idn : id;
                                    const uint32_t dt = tmem + (uint32_t)(co * NP);
                                    // the first product into each accumulator overwrites it
                                    const uint32_t en = (ci | pr | ks) ? 1u : first;
                                    if (C::ATM) {
                                        // A from tensor memory: block ablk, K step ks (8 columns per MMA)
                                        const uint32_t ta = tmem + kAcol + (uint32_t)ablk * Lt::ACOLS + 8u * ks;
                                        if (C::FMT == 2)
                                            asm volatile(
                                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                                "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dt),
                                                "r"(ta), "l"(db), "r"(idd), "r"(en));
                                        else
                                            asm volatile(
                                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                                "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dt),
                                                "r"(ta), "l"(db), "r"(idd), "r"(en));
                                    } else {
                                        const uint64_t da = dAs + (uint64_t)((ablk * Lt::ABLK + 256 * ks) >> 4);
                                        if (C::FMT == 2)
                                            asm volatile(
                                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                                                "l"(da), "l"(db), "r"(idd), "r"(en));
                                        else
                                            tc::mma_bf16(dt, da, db, idd, en);
                                    }
                                }
                    if (C::ATM) tc::commit(&aempty);
                    tc::commit(&empty[s]);
                }
                tc::commit(&done);  // also after a stop: fires once the issued products are complete
            }
        } else {
            // ---- builders (warps 0..7) ----
            const int tid = threadIdx.x;                  // 0 .. 255
            const int a_loc = (warp & 3) * 32 + lane;     // TMEM lane = GEMM row
            const int hb = warp >> 2;                     // which 8 of the stage's 16 columns
            const int a = tA * kRows + a_loc;
            const int2 xa = A.xy_p[a];
            const int4 bA = A.bbox_a[tA];
            const float* tk = A.tab32 + (size_t)(k - A.kbase) * A.Dy * A.Dx * 6;
            // table sub-box and interface offsets of tile tB into buffer buf, by asynchronous copies
            auto stage_async = [&](int buf, int tB) {
                const int4 bB = A.bbox_b[tB];
                const int ox = bA.x - bB.y, oy = bA.z - bB.w;
                float* dt = s_tab + (size_t)buf * HW * 6;
                for (int e = tid; e < HW; e += kBuilders) {
                    const int iy = e / A.W, ix = e - iy * A.W;
                    const int gx = ox + ix - A.box_x0, gy = oy + iy - A.box_y0;
                    const bool in = gx < A.Dx && gy < A.Dy;
                    const float* src = in ? tk + ((size_t)gy * A.Dx + gx) * 6 : tk;  // zero fill outside the box
#pragma unroll
                    for (int h = 0; h < 3; h++) cp_async8(dt + (size_t)e * 6 + 2 * h, src + 2 * h, in ? 8 : 0);
                }
                if (tid < kTileB / 4) cp_async16(s_off + buf * kTileB + 4 * tid, A.off_i + tB * kTileB + 4 * tid);
                asm volatile("cp.async.commit_group;" ::: "memory");
            };
            // Accumulators -> uh32 (the modes k >= 1 in FP32).  The FP32 accumulation in tensor
            // memory truncates at every step, so the interface sum is split into groups of gs
            // stages whose partial sums are added here with round-to-nearest FP32 adds; the first
            // group writes, the later ones add.  The sums are FP32 values, kept in FP32.
            const uint32_t tacc = tmem + ((uint32_t)((warp & 3) * 32) << 16);
            auto drain = [&](bool add) {
                for (int c0 = hb * 16; c0 < NP; c0 += 32) {
                    float v0[16], v1[16], v2[16];
                    tc::ld16(tacc + (uint32_t)c0, v0);
                    tc::ld16(tacc + (uint32_t)(NP + c0), v1);
                    tc::ld16(tacc + (uint32_t)(2 * NP + c0), v2);
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        // four right-hand sides at a time: every load issued before any store
                        float2 q[4][3];
                        float2* o[4];
#pragma unroll
                        for (int jj = 0; jj < 4; jj++) {
                            const int r = c0 / 2 + h * 4 + jj;
                            o[jj] = (float2*)(A.uh32 + (((size_t)(r0 + min(r, RG - 1)) * A.K + k) * A.NPpad + a) * 6);
                            if (add && r < RG) q[jj][0] = o[jj][0], q[jj][1] = o[jj][1], q[jj][2] = o[jj][2];
                        }
#pragma unroll
                        for (int jj = 0; jj < 4; jj++) {
                            const int j = h * 4 + jj, r = c0 / 2 + j;
                            if (r >= RG) continue;
                            float w[6] = {v0[2 * j], v1[2 * j], v2[2 * j], v0[2 * j + 1], v1[2 * j + 1], v2[2 * j + 1]};
                            if (add) {
                                w[0] += q[jj][0].x, w[1] += q[jj][0].y, w[2] += q[jj][1].x;
                                w[3] += q[jj][1].y, w[4] += q[jj][2].x, w[5] += q[jj][2].y;
                            }
                            o[jj][0] = make_float2(w[0], w[1]);
                            o[jj][1] = make_float2(w[2], w[3]);
                            o[jj][2] = make_float2(w[4], w[5]);
                        }
                    }
                }
            };
            int il = 0, gpos = 0;  // stage of the item and its position in the accumulation group
            if (nbuf == 2) stage_async(0, 0);
            for (int tB = 0; tB < A.n_tb; tB++) {
                if (nbuf == 1) {
                    if (builders_sync_any(s_abort)) break;  // everyone is done with the previous tile
                    stage_async(0, tB);
                }
                asm volatile("cp.async.wait_all;" ::: "memory");
                // this tile's copies are visible to every builder, the previous tile is done;
                // the same stop decision in every builder
                if (builders_sync_any(s_abort)) break;
                if (nbuf == 2 && tB + 1 < A.n_tb) stage_async((tB + 1) & 1, tB + 1);
                const int buf = nbuf == 2 ? (tB & 1) : 0;
                const float* tab_b = s_tab + (size_t)buf * HW * 6;
                const int* off_b = s_off + buf * kTileB;
                const int4 bB = A.bbox_b[tB];
                const int ox = bA.x - bB.y, oy = bA.z - bB.w;
                const int base = (xa.x - ox) + A.W * (xa.y - oy);
                for (int st = 0; st < kStagesPerTile; st++, il++) {
                    const uint32_t it = it_base + il;
                    const int s = it % S;
                    const uint32_t u = it / S;
                    if (!C::ATM && (s_abort || !wait_or_abort(&empty[s], (u & 1u) ^ 1u, &s_abort, wl))) {
                        s_abort = 1;
                        continue;  // keep the barrier count of the other builders
                    }
                    // At a group boundary, wait for the previous stage's products first (A in tensor
                    // memory: the A buffer's release; otherwise the single stage's release above)
                    // and drain the accumulators before gathering, where few registers are live.
                    bool drained = false;
                    const bool boundary = il > 0 && gpos == 0;
                    if (++gpos == gs) gpos = 0;
                    if (boundary) {
                        if (C::ATM && (s_abort || !wait_or_abort(&aempty, (it & 1u) ^ 1u, &s_abort, wl))) {
                            s_abort = 1;
                            continue;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        drain(il > gs);
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        drained = true;
                    }
                    // row a_loc, columns st*16 + hb*8 .. + 7 of this tile: six entries, NS pieces each
                    float v[8][6];
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const int idx = base - off_b[st * kKC + hb * 8 + i];
                        const float2* src = (const float2*)(tab_b + (size_t)idx * 6);
                        const float2 p0 = src[0], p1 = src[1], p2 = src[2];
                        v[i][0] = p0.x, v[i][1] = p0.y, v[i][2] = p1.x, v[i][3] = p1.y, v[i][4] = p2.x, v[i][5] = p2.y;
                    }
                    // split into NS pieces: four 32-bit words (eight bf16, or four tf32 twice) per entry and piece
                    uint32_t wq[6][C::NS][4], wt[6][2][4];
#pragma unroll
                    for (int e = 0; e < 6; e++) {
                        float x[8];
#pragma unroll
                        for (int i = 0; i < 8; i++) x[i] = v[i][e];
                        if (C::ES == 2) {
                            // bf16 pieces two at a time: packed round-to-nearest conversion, exact FP32 remainders
#pragma unroll
                            for (int p = 0; p < C::NS; p++)
#pragma unroll
                                for (int i = 0; i < 4; i++) {
                                    uint32_t w;
                                    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(x[2 * i + 1]), "f"(x[2 * i]));
                                    wq[e][p][i] = w;
                                    if (p + 1 < C::NS) {
                                        x[2 * i] = __fsub_rn(x[2 * i], __uint_as_float(w << 16));
                                        x[2 * i + 1] = __fsub_rn(x[2 * i + 1], __uint_as_float(w & 0xffff0000u));
                                    }
                                }
                        } else {
#pragma unroll
                            for (int q = 0; q < 2; q++)
#pragma unroll
                                for (int i = 0; i < 4; i++) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(wt[e][q][i]) : "f"(x[4 * q + i]));
                        }
                    }
                    if (C::ATM) {
                        // the tensor-memory A buffer is free once the previous stage's products are complete
                        if (!drained && (s_abort || !wait_or_abort(&aempty, (it & 1u) ^ 1u, &s_abort, wl))) {
                            s_abort = 1;
                            continue;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        // lane = row a_loc; columns: block * ACOLS + this thread's K half
                        const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + kAcol;
#pragma unroll
                        for (int e = 0; e < 6; e++) {
                            if (C::ES == 2) {
#pragma unroll
                                for (int p = 0; p < C::NS; p++)
                                    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                                                     trow + (uint32_t)(e * C::NS + p) * Lt::ACOLS + 4u * hb),
                                                 "r"(wq[e][p][0]), "r"(wq[e][p][1]), "r"(wq[e][p][2]), "r"(wq[e][p][3])
                                                 : "memory");
                            } else {
                                asm volatile(
                                    "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
                                        trow + (uint32_t)e * Lt::ACOLS + 8u * hb),
                                    "r"(wt[e][0][0]), "r"(wt[e][0][1]), "r"(wt[e][0][2]), "r"(wt[e][0][3]), "r"(wt[e][1][0]),
                                    "r"(wt[e][1][1]), "r"(wt[e][1][2]), "r"(wt[e][1][3])
                                    : "memory");
                            }
                        }
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&afull);
                    } else {
                        unsigned char* dstA = sA + s * Lt::A_STAGE;
#pragma unroll
                        for (int e = 0; e < 6; e++) {
                            if (C::ES == 2) {
#pragma unroll
                                for (int p = 0; p < C::NS; p++) {
                                    const uint32_t off = (uint32_t)(a_loc / 8) * Lt::SBO + hb * 128 + (a_loc % 8) * 16;
                                    *(uint4*)(dstA + (size_t)(e * C::NS + p) * Lt::ABLK + off) =
                                        make_uint4(wq[e][p][0], wq[e][p][1], wq[e][p][2], wq[e][p][3]);
                                }
                            } else {
#pragma unroll
                                for (int q = 0; q < 2; q++) {
                                    const int kc = hb * 2 + q;
                                    const uint32_t off = (uint32_t)(a_loc / 8) * Lt::SBO + kc * 128 + (a_loc % 8) * 16;
                                    *(uint4*)(dstA + (size_t)e * Lt::ABLK + off) =
                                        make_uint4(wt[e][q][0], wt[e][q][1], wt[e][q][2], wt[e][q][3]);
                                }
                            }
                        }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&full[s]);
                    }
                }
            }
            asm volatile("cp.async.wait_all;" ::: "memory");  // a prefetch still in flight after a stop
            // ---- epilogue: accumulators -> uh (FP64) ----
            // the MMA thread commits `done` once per item on every path, also after a stop; every product it
            // issued is complete once `done` fires, so this wait keeps the full bound whatever the stop flag says
            const bool done_ok = tc::mbar_wait(&done, n_done & 1u);
            const bool ok = done_ok && !s_abort;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (ok) drain(n_it > gs);  // the last group; earlier groups were drained in the loop
        }
    }
}

template <int PREC>
__device__ __forceinline__ void tc_setup(TcSync<TcCfg<PREC>::S>& sy) {
    constexpr int S = TcCfg<PREC>::S;
    if (threadIdx.x == 0) {
        sy.abort = 0;
        for (int s = 0; s < S; s++) mbar_init(&sy.full[s], kBuilderWarps), mbar_init(&sy.bfull[s], 1), mbar_init(&sy.empty[s], 1);
        mbar_init(&sy.done, 1);
        mbar_init(&sy.afull, kBuilderWarps), mbar_init(&sy.aempty, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x / 32 == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sy.tbase)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <int PREC>
__device__ __forceinline__ void tc_teardown(TcSync<TcCfg<PREC>::S>& sy, int* status) {
    __syncthreads();
    if (threadIdx.x == 0 && sy.abort) atomicExch(status, FBC_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x / 32 == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sy.tbase), "r"(kTmemCols));
}

// One plan: one item per CTA from its grid position (pad tile, mode k0 + y, rhs group).
template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) k_contract_tc(TcJob J, int wl, int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ TcSync<TcCfg<PREC>::S> sy;
    tc_setup<PREC>(sy);
    tc_item<PREC>(J, make_int4(0, J.A.k0 + (int)blockIdx.y, (int)blockIdx.x, (int)blockIdx.z), 0u, 0u, sy, smem, wl);
    tc_teardown<PREC>(sy, status);
}

// A batch of plans: persistent CTAs take items (job, k, pad tile, rhs group) from a queue with atomicAdd; no
// CTA waits for another.  The stage counters and barrier phases run on across items, so no barrier is
// re-initialised while a tensor-core commit could still arrive on it; the CTA-wide barrier between items
// orders the drain of one item's accumulators before the next item's first products.
template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    k_contract_tc_queue(const TcJob* __restrict__ jobs, const int4* __restrict__ items, int n_items,
                        int* __restrict__ counter, int wl, int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ TcSync<TcCfg<PREC>::S> sy;
    __shared__ int s_item;
    __shared__ int4 s_wk;
    __shared__ TcJob s_job;  // the current item's job
    tc_setup<PREC>(sy);
    uint32_t it_base = 0, n_done = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int ii = atomicAdd(counter, 1);
            s_item = ii;
            if (ii < n_items) s_wk = items[ii], s_job = jobs[s_wk.x];
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (s_item >= n_items || sy.abort) break;
        tc_item<PREC>(s_job, s_wk, it_base, n_done, sy, smem, wl);
        it_base += (uint32_t)(s_job.A.n_tb * kStagesPerTile);
        n_done++;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // every role is done with s_job and s_wk before thread 0 overwrites them
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    tc_teardown<PREC>(sy, status);
}

template <int PREC>
size_t tc_smem(int HW, int nbuf) {
    using Lt = TcLayout<PREC>;
    return TcCfg<PREC>::S * (Lt::A_STAGE + Lt::B_STAGE) + nbuf * ((size_t)6 * HW * 4 + (size_t)kTileB * 4) + 1024;
}
// two table buffers (the next tile prefetched) when they fit, else one
template <int PREC>
int tc_nbuf(int HW) { return tc_smem<PREC>(HW, 2) <= 227 * 1024 ? 2 : 1; }
template <int PREC>
size_t tc_smem(int HW) { return tc_smem<PREC>(HW, tc_nbuf<PREC>(HW)); }

int prep_groups(const Plan& P) { return (P.opt.max_rhs + kRhsPerCta - 1) / kRhsPerCta; }
int prep_rows(const Plan& P) { return ((2 * std::min(kRhsPerCta, P.opt.max_rhs) + 15) / 16) * 16; }
int rows_for(int rpc) { return ((2 * rpc + 15) / 16) * 16; }

template <int PREC>
size_t prep_bytes(const Plan& P) {
    using C = TcCfg<PREC>;
    return (size_t)P.K * prep_groups(P) * P.n_tb * kStagesPerTile * 3 * C::NS * prep_rows(P) * kKC * C::ES;
}

// Split the force operand of modes k0 .. k0 + n_modes - 1 into the plan's buffer, rpc right-hand sides per group.
template <int PREC>
cudaError_t prep_tc(const Plan& P, const double* fh, int rpc, int n_rhs, int k0, int n_modes, cudaStream_t st) {
    using Lt = TcLayout<PREC>;
    const int G = (P.opt.max_rhs + rpc - 1) / rpc, npb = rows_for(rpc);
    const size_t total = (size_t)n_modes * G * P.n_tb * kStagesPerTile * 3 * npb * (kKC / Lt::KPC);
    const int grid = (int)std::min<size_t>((total + 255) / 256, (size_t)152 * 32);
    k_prep_b<PREC><<<grid, 256, 0, st>>>(fh, P.K, P.NIpad, P.n_tb, G, npb, rpc, n_rhs, k0, n_modes,
                                         (unsigned char*)P.d_bprep);
    return cudaGetLastError();
}

template <int PREC>
TcJob make_job(const ContractArgs& A, const Plan& P, int n_rhs, int rpc, int nbuf) {
    TcJob J;
    J.A = A;
    J.bprep = (const unsigned char*)P.d_bprep;
    J.n_rhs = n_rhs;
    J.rpc = rpc;
    J.G = (P.opt.max_rhs + rpc - 1) / rpc;
    J.npb = rows_for(rpc);
    // accumulation groups of kDrainTiles interface tiles (1024 columns), or one group
    const int n_it = P.n_tb * kStagesPerTile;
    J.gs = (P.opt.flags & FBC_PLAN_TC_FAST_ACCUMULATE) ? n_it : std::min(n_it, kDrainTiles * kStagesPerTile);
    J.nbuf = nbuf;
    return J;
}

template <int PREC>
cudaError_t launch_tc(const ContractArgs& A, const Plan& P, int n_rhs, cudaStream_t st, int n_modes) {
    const size_t smem = tc_smem<PREC>(P.H * P.W);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    if (!P.d_bprep || P.bprep_prec != PREC || n_rhs > P.opt.max_rhs) return cudaErrorInvalidValue;
    const int rpc = std::min(kRhsPerCta, P.opt.max_rhs);
    if (cudaError_t e = prep_tc<PREC>(P, A.fh, rpc, n_rhs, A.k0, n_modes, st)) return e;
    cudaError_t e = cudaFuncSetAttribute(k_contract_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    const TcJob J = make_job<PREC>(A, P, n_rhs, rpc, tc_nbuf<PREC>(P.H * P.W));
    dim3 grid(P.n_ta, n_modes, (n_rhs + rpc - 1) / rpc);
    const int wl = P.wait_limit > 0 ? P.wait_limit : tc::kWaitLimit;
    k_contract_tc<PREC><<<grid, kThreads, smem, st>>>(J, wl, P.d_status);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_tc_batch(const TcJob* d_jobs, const int4* d_items, int n_items, int* d_counter, int grid,
                            size_t smem, int wl, int* status, cudaStream_t st) {
    cudaError_t e =
        cudaFuncSetAttribute(k_contract_tc_queue<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    k_contract_tc_queue<PREC><<<grid, kThreads, smem, st>>>(d_jobs, d_items, n_items, d_counter, wl, status);
    return cudaGetLastError();
}

}  // namespace

size_t contract_tc_smem(int precision, int HW) {
    if (precision == FBC_PREC_TF32) return tc_smem<FBC_PREC_TF32>(HW);
    if (precision == FBC_PREC_BF16X2) return tc_smem<FBC_PREC_BF16X2>(HW);
    return tc_smem<FBC_PREC_BF16X3>(HW);
}

size_t contract_tc_prep_bytes(const Plan& P, int precision) {
    if (precision == FBC_PREC_TF32) return prep_bytes<FBC_PREC_TF32>(P);
    if (precision == FBC_PREC_BF16X2) return prep_bytes<FBC_PREC_BF16X2>(P);
    return prep_bytes<FBC_PREC_BF16X3>(P);
}

// Largest rhs group a plan's force-operand buffer holds (right-hand sides per CTA), and whether rpc fits it:
// the buffer holds G x npb rows per (mode, stage) for the plan's own group size.
int contract_tc_max_rpc(const Plan& P) { return std::min(kRhsPerCta, P.opt.max_rhs); }
bool contract_tc_rpc_fits(const Plan& P, int rpc) {
    if (rpc < 1 || rpc > contract_tc_max_rpc(P)) return false;
    const long long want = (long long)((P.opt.max_rhs + rpc - 1) / rpc) * rows_for(rpc);
    return want <= (long long)prep_groups(P) * prep_rows(P);
}

size_t contract_tc_nbuf_smem(int precision, int HW, int nbuf) {
    if (precision == FBC_PREC_TF32) return tc_smem<FBC_PREC_TF32>(HW, nbuf);
    if (precision == FBC_PREC_BF16X2) return tc_smem<FBC_PREC_BF16X2>(HW, nbuf);
    return tc_smem<FBC_PREC_BF16X3>(HW, nbuf);
}

cudaError_t contract_tc_prep(const Plan& P, const double* fh, int rpc, int n_rhs, int k0, int n_modes, cudaStream_t st) {
    if (!P.d_bprep || P.bprep_prec != P.precision || !contract_tc_rpc_fits(P, rpc)) return cudaErrorInvalidValue;
    if (P.precision == FBC_PREC_TF32) return prep_tc<FBC_PREC_TF32>(P, fh, rpc, n_rhs, k0, n_modes, st);
    if (P.precision == FBC_PREC_BF16X2) return prep_tc<FBC_PREC_BF16X2>(P, fh, rpc, n_rhs, k0, n_modes, st);
    if (P.precision == FBC_PREC_BF16X3) return prep_tc<FBC_PREC_BF16X3>(P, fh, rpc, n_rhs, k0, n_modes, st);
    return cudaErrorInvalidValue;
}

TcJob contract_tc_job(const Plan& P, int n_rhs, int rpc, int nbuf) {
    const ContractArgs A = make_contract_args(P);
    if (P.precision == FBC_PREC_TF32) return make_job<FBC_PREC_TF32>(A, P, n_rhs, rpc, nbuf);
    if (P.precision == FBC_PREC_BF16X2) return make_job<FBC_PREC_BF16X2>(A, P, n_rhs, rpc, nbuf);
    return make_job<FBC_PREC_BF16X3>(A, P, n_rhs, rpc, nbuf);
}

cudaError_t launch_contract_tc_batch(int precision, const TcJob* d_jobs, const int4* d_items, int n_items,
                                     int* d_counter, int grid, size_t smem, int wl, int* status, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    if (precision == FBC_PREC_TF32)
        return launch_tc_batch<FBC_PREC_TF32>(d_jobs, d_items, n_items, d_counter, grid, smem, wl, status, st);
    if (precision == FBC_PREC_BF16X2)
        return launch_tc_batch<FBC_PREC_BF16X2>(d_jobs, d_items, n_items, d_counter, grid, smem, wl, status, st);
    if (precision == FBC_PREC_BF16X3)
        return launch_tc_batch<FBC_PREC_BF16X3>(d_jobs, d_items, n_items, d_counter, grid, smem, wl, status, st);
    return cudaErrorInvalidValue;
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
