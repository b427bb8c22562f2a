// Internal declarations of the FBC pad-update library (not part of the ABI).
//
// Data layout in device memory (FP64 unless noted):
//   f   [n_rhs][n_i][L][3]        caller's interface forces (original column order)
//   u   [n_rhs][n_p][L][3]        caller's pad displacements
//   fh  [max_rhs][K][NIpad][6]    forward transform of f, tile-sorted columns
//   uh  [max_rhs][K][NPpad][6]    contracted modes, tile-sorted pad columns
//   tab [K][Dy][Dx][6]            mode table g^k(d), d = (box_x0 + ix, box_y0 + iy)
// with K = L/2 + 1.  A "six-vector" of a complex 3-vector V is
//   (Re V1, Re V2, Im V3, Im V1, Im V2, -Re V3):
// the first half is x, the second half y'.  For a mirror-symmetric medium the
// per-mode 3x3 block is  g = A + iB  with A even (11, 12, 22, 33) and B odd
// (13, 23), and U = g F becomes the same real 3x3 matrix
//   M = [[A11, A12, -B13], [A12, A22, -B23], [B13, B23, A33]]
// acting on x and on y' separately (two real right-hand sides per mode).
// The table stores (A11, A12, A22, A33, B13, B23).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "fbc.h"
#include "fbc_fft.cuh"

namespace fbc {

constexpr int kMaxRichImages = 40;  // n + N upper bound
constexpr int kMaxQuad = 512;       // Barnett nodes on [0, pi)
constexpr int kHostChunks = 8;      // host-memory apply: right-hand-side chunks at most
constexpr int kHostChunkRhs = 4;    // ... and right-hand sides per chunk at least
constexpr int kTileA = 128;         // pad columns per contraction tile
constexpr int kTileB = 64;          // interface columns per contraction tile
// Private bit of Plan::opt.flags, above every FBC_PLAN_* bit: set by
// fbc_plan_lattice_near_field once the near field is in the table, cleared by
// a new tabulation; applies of a plan with FBC_PLAN_SELF_TERMS need it.
constexpr int kPlanNearFieldSet = 1 << 30;

// Material constants as the tabulation kernels read them.
struct MaterialDev {
    int kind;          // FBC_MATERIAL_*
    double kelvin_pre; // 1 / (16 pi mu (1 - nu))
    double kelvin_a;   // 3 - 4 nu
    double K[36];      // Christoffel form: M_I = sum_J K[I][J] zz_J, I, J over symmetric pairs
    int nquad;
};

struct TabulateParams {
    int L, K, Lh;           // Lh = L / 2
    double c;
    int rich_n, rich_N;
    double W[kMaxRichImages];  // cumulative Richardson weights of images n+1 .. n+N
    int box_x0, box_y0, Dx, Dy;
};

struct FftGrid;  // in-plane FFT form (fbc_fft2d.cu)

struct Plan {
    int device = 0;
    int n_i = 0, n_p = 0, L = 0, K = 0, logL = 0;
    double c = 1.0;
    int TA = kTileA, TB = kTileB;
    int n_ta = 0, n_tb = 0, NIpad = 0, NPpad = 0;
    int box_x0 = 0, box_y0 = 0, Dx = 0, Dy = 0;  // difference table box
    int W = 0, H = 0;                             // largest tile-pair sub-box
    int n_used = 0;
    fbc_options opt{};
    MaterialDev mat{};
    TabulateParams tp{};
    bool tabulated = false;
    int precision = FBC_PREC_FP64;

    // host copies of the sorted layout
    std::vector<int> perm_i, perm_p;  // sorted slot -> original column (-1 = padding)
    std::vector<int2> xy_i_sorted, xy_p_sorted;
    bool host_only = false;

    // device buffers (owned)
    int2* d_xy_p = nullptr;      // [NPpad] sorted pad sites (padding: first site of its tile)
    int* d_off_i = nullptr;      // [NIpad] x_b + W * y_b of the sorted interface sites
    int4* d_bbox_a = nullptr;    // [n_ta] (minx, maxx, miny, maxy)
    int4* d_bbox_b = nullptr;    // [n_tb]
    int* d_perm_i = nullptr;     // [NIpad]
    int* d_perm_p = nullptr;     // [NPpad]
    int2* d_used = nullptr;      // [n_used] differences that occur
    double2* d_tw = nullptr;     // [L/2] exp(-2 pi i t / L), then the same as [L/2] float2
    double2* d_twL = nullptr;    // [L] (cos, sin)(2 pi t / L) for the table DFT
    float2* d_twl = nullptr;     // [L] exp(-2 pi i t / L) in FP32: the Stockham FP32 line transforms
    Fft1D line_fft;              // their passes (length L)
    double* d_table = nullptr;   // [K][Dy][Dx][6] FP64
    float* d_table32 = nullptr;  // [K][Dy][Dx][6] FP32 (FBC_PREC_FP32)
    float* d_table_x2 = nullptr; // [K][Dy][Dx][12] hi/lo pairs (FBC_PREC_F32X2)
    float* d_table_x2_k0 = nullptr; // [Dy][Dx][12]: the k = 0 slice as hi/lo pairs (FP32 and tensor-core plans)
    double* d_fh = nullptr;      // [max_rhs][K][NIpad][6]
    double* d_uh = nullptr;      // [max_rhs][K][NPpad][6]
    float* d_uh32 = nullptr;     // [max_rhs][K][NPpad][6]: the modes k >= 1 of the tensor-core forms (FP32 sums)
    double* d_part = nullptr;    // [max_rhs][n_line_blocks_p][3] zero-mean partial sums
    double* d_relax = nullptr;   // [max_rhs][kRelaxBlocks][2] dot products, then [max_rhs][n_line_blocks_p] maxima
    double* d_stage_f = nullptr; // host-apply staging
    double* d_stage_u = nullptr;
    int* d_status = nullptr;     // device error word
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // stage timing (optional)
    // host-memory apply: copy-in and copy-out streams and their events (created on first use)
    cudaStream_t host_st[2] = {nullptr, nullptr};
    cudaEvent_t host_ev[2 * kHostChunks + 2] = {};
    // learned far field (fbc_plan_attach_surrogate): streamed per-mode slices
    fbc_surrogate* sur = nullptr;
    double sur_rmin = 0.0;
    size_t sur_bytes = 0;
    bool tables_released = false;
    int n_far = 0, n_near = 0;
    int2* d_far = nullptr;
    int2* d_near = nullptr;
    float* d_near32 = nullptr;   // [K][n_near][6] exact entries of the near field
    float* d_slice = nullptr;    // [sur_chunk][Dy][Dx][6] streamed mode slices (FP32)
    int sur_chunk = 0;           // modes per streamed chunk
    // tensor-core forms: the force operand split once per apply (fbc_contract_tc.cu)
    void* d_bprep = nullptr;
    size_t bprep_bytes = 0;
    int bprep_prec = -1;
    int wait_limit = 0;  // polls per pipeline wait of the tensor-core contraction (0: the default bound)
    bool timing = false, timed_once = false;
    size_t table_bytes = 0, workspace_bytes = 0;
    FftGrid* fft = nullptr;  // in-plane FFT form: grid, transformed kernel, workspace
};

// Everything a contraction tile needs about one plan (one instance of a batch).
struct ContractArgs {
    const double* tab;   // [K][Dy][Dx][6]
    const float* tab32;  // [K][Dy][Dx][6]
    const float* tabx2;  // [K][Dy][Dx][12] (hi, lo) pairs of the six reals
    const double* fh;    // [rhs][K][NIpad][6]
    double* uh;          // [rhs][K][NPpad][6]
    float* uh32;         // [rhs][K][NPpad][6] the tensor-core forms' modes k >= 1
    const int2* xy_p;
    const int* off_i;
    const int4* bbox_a;
    const int4* bbox_b;
    int n_tb, K, Dx, Dy, box_x0, box_y0, W, H, NIpad, NPpad, k0;
    int kbase;  // the tables hold mode slices kbase, kbase + 1, ... (0: all K; else a streamed chunk)
    int* status;  // device error word (a bounded wait that gave up)
};

// One instance's share of a tensor-core contraction launch (fbc_contract_tc.cu).
struct TcJob {
    ContractArgs A;
    const unsigned char* bprep;  // split force operand: chunks (mode, rhs group, interface tile, stage)
    int n_rhs;                   // right-hand sides applied
    int rpc;                     // right-hand sides per CTA (one rhs group)
    int G;                       // rhs groups in the operand buffer's layout
    int npb;                     // force-operand rows per chunk: 2 rpc rounded up to 16
    int gs;                      // stages per tensor-memory accumulation group
    int nbuf;                    // table sub-box buffers in shared memory (2: the next tile prefetched)
};

// Everything the line transforms need about one plan (one instance of a batch).
struct LineArgs {
    Fft1D F;           // Stockham passes of length L (FP32 forms)
    const float2* twl; // their twiddles
    int stockham;      // 1: FP32 transforms in the Stockham form (L <= kLineStockhamMaxL, 16-byte aligned arrays)
    const float* uh32; // the tensor-core forms' modes k >= 1 in FP32 (nullptr: every mode in uh)
    const double* f;   // caller forces [n_rhs][n_i][L][3]
    double* u;         // caller displacements [n_rhs][n_p][L][3]
    double* fh;
    double* uh;
    const int* perm_i;
    const int* perm_p;
    const double2* tw;
    double* part;
    int n_i, n_p, L, logL, K, NIpad, NPpad, NC;
};

// ---- launchers (each returns the launch's cudaError_t) ---------------------
cudaError_t launch_tabulate(Plan& P, cudaStream_t st);
// The periodic kernel in real space, G~(d, s) for s = 0..L/2 (the stage before the line DFT), as
// FP32 six-entry records at every cell of the difference box: out[Dy * Dx][L/2 + 1][6] (11, 12, 22,
// 33, 13, 23); cells of differences that do not occur are zero.  The H-matrix build reads it.
cudaError_t launch_real_space_table(Plan& P, float* out, cudaStream_t st);
cudaError_t launch_forward(Plan& P, const double* f, int n_rhs, bool project, cudaStream_t st);
cudaError_t launch_contract(Plan& P, int n_rhs, cudaStream_t st);
// alpha_dev (optional): per-rhs multiplier alpha_dev_scale * alpha_dev[r] in place of alpha / L;
// gmax_part (optional): only record per (rhs, line block) the largest |value|, write nothing
cudaError_t launch_inverse(Plan& P, double* u, int n_rhs, double alpha, double beta, bool zero_mean,
                           cudaStream_t st, const double* alpha_dev = nullptr, double alpha_dev_scale = 0.0,
                           double* gmax_part = nullptr);
// residual-based relaxation (fbc_relax.cu)
constexpr int kRelaxBlocks = 128;  // blocks per right-hand side of the dot-product pass
cudaError_t launch_relax_dots(const double* f_new, const double* f_old, size_t n_per_rhs, int n_rhs, double* part,
                              cudaStream_t st);
cudaError_t launch_relax_alpha(const double* dot_part, int has_old, const double* gmax_part, int n_gblk, int n_rhs,
                               double du_max, double* alpha_io, cudaStream_t st);
cudaError_t launch_derive_tables(Plan& P, int precision, cudaStream_t st);
// in-plane FFT form (fbc_fft2d.cu): host structures and buffers (once; needs the uploaded difference
// list), the grid's transformed kernel from the FP64 table, the contraction, release
int fft_prepare(Plan& P, int precision);
bool fft_ready(const Plan& P, int precision);
cudaError_t launch_fft_tables(Plan& P, int precision, cudaStream_t st);
cudaError_t launch_contract_fft(Plan& P, int n_rhs, cudaStream_t st);
void fft_free(Plan& P);
void fft_info(const Plan& P, int* mx, int* my, int* rows_i, int* rows_p, int* chunk_items);
ContractArgs make_contract_args(const Plan& P);
cudaError_t launch_contract_tc(const ContractArgs& A, const Plan& P, int n_rhs, cudaStream_t st, int n_modes = -1);
// contraction of modes k0 .. k0 + n_modes - 1 in the plan's precision (k0 >= 1 for the FP32 and tensor forms)
cudaError_t launch_contract_modes(Plan& P, const ContractArgs& A, int k0, int n_modes, int n_rhs, cudaStream_t st);
cudaError_t launch_contract_x2_k0(Plan& P, const ContractArgs& A, int n_rhs, cudaStream_t st);
// streamed contraction of a plan with an attached surrogate (modes k >= 1)
cudaError_t launch_contract_streamed(Plan& P, int n_rhs, cudaStream_t st);
void release_surrogate_buffers(Plan& P);
size_t contract_tc_smem(int precision, int HW);
size_t contract_tc_nbuf_smem(int precision, int HW, int nbuf);
size_t contract_tc_prep_bytes(const Plan& P, int precision);
// tensor-core batches: rhs groups a plan's operand buffer holds, the split of one instance's forces, its job
// record, and the persistent launch over a queue of items (job, k, pad tile, rhs group)
int contract_tc_max_rpc(const Plan& P);
bool contract_tc_rpc_fits(const Plan& P, int rpc);
cudaError_t contract_tc_prep(const Plan& P, const double* fh, int rpc, int n_rhs, int k0, int n_modes, cudaStream_t st);
TcJob contract_tc_job(const Plan& P, int n_rhs, int rpc, int nbuf);
cudaError_t launch_contract_tc_batch(int precision, const TcJob* d_jobs, const int4* d_items, int n_items,
                                     int* d_counter, int grid, size_t smem, int wl, int* status, cudaStream_t st);
// FBC_PREC_BF16X6 (fbc_contract_oz.cu): shared memory of the contraction, bytes of the sliced force
// operand and scales (the plan's d_bprep), and the launch of modes A.k0 .. K - 1
size_t contract_oz_smem(int HW);
size_t contract_oz_prep_bytes(const Plan& P);
int contract_oz_rhs_group();  // right-hand sides per CTA
cudaError_t launch_contract_oz(const ContractArgs& A, const Plan& P, int n_rhs, cudaStream_t st);
inline bool is_tensor_precision(int p) { return p == FBC_PREC_TF32 || p == FBC_PREC_BF16X2 || p == FBC_PREC_BF16X3; }
int batch_rhs_block();
LineArgs make_line_args(const Plan& P, const double* f, double* u);
// dynamic shared memory of one instance's batched line transforms (FP64 or FP32 form; a batch launches
// with the largest over its instances)
size_t line_args_smem(const LineArgs& A, bool fp32);
// stage 0 forward, 1 projection, 2 inverse, 3 zero mean; items as documented in fbc_line.cu
cudaError_t launch_batch_line(int stage, const LineArgs* d_args, const int4* d_items, int n_items, size_t smem,
                              double alpha, double beta, int want_part, cudaStream_t st, bool fp32);
// line transforms in FP32 (k = 0 kept in FP64) for the FP32 and tensor-core contractions
inline bool is_fft_precision(int p) { return p == FBC_PREC_FFT64 || p == FBC_PREC_FFT32; }
inline bool line_fp32(int precision) {
    return precision == FBC_PREC_FP32 || is_tensor_precision(precision) || precision == FBC_PREC_FFT32;
}
// phase 0: k = 0 items (double-float tile), phase 1: k >= 1 items of an FP32 batch (8-rhs FP32 tile);
// FP64 and double-float batches use phase 1 with their own tile for every item
cudaError_t launch_batch_contract(int precision, int phase, const ContractArgs* d_args, const int* d_n_rhs,
                                  const int4* d_items, int n_items, int* d_counter, int grid, size_t smem,
                                  cudaStream_t st);
size_t batch_contract_smem_phase(int precision, int phase, int W, int H);
int batch_contract_occupancy_phase(int precision, int phase, size_t smem);

// ---- learned surrogate of the mode table (fbc_surrogate.cu, fbc_mlp_tc.cu) ----
constexpr int kSurIn = 4, kSurOut = 6;
// beyond q r = kQrCut a k >= 1 entry is served as zero (and never trained on)
constexpr double kQrCut = 16.0;

// Network inputs of difference d (d != 0) at mode k >= 1:
// (ln(q r) / 4, d_x / r, d_y / r, ln(r) / 5) with q = 2 pi k / (L c); returns q r.
__host__ __device__ inline double surrogate_features(int dx, int dy, int k, int L, double c, float* x) {
    const double r = sqrt((double)dx * dx + (double)dy * dy);
    const double qr = 2.0 * 3.14159265358979323846 * k / (L * c) * r;
    x[0] = (float)(log(qr) * 0.25);
    x[1] = (float)(dx / r);
    x[2] = (float)(dy / r);
    x[3] = (float)(log(r) * 0.2);
    return qr;
}
// s(q, r) = exp(-q r) / (c sqrt(1 + q r)), zero beyond the cut
__host__ __device__ inline double surrogate_scale(double qr, double c) {
    return qr > kQrCut ? 0.0 : exp(-qr) / (c * sqrt(1.0 + qr));
}

// Fused tensor-core inference (fbc_mlp_tc.cu).  Rows are either given as
// features (X [n][4] -> Y [n][6]) or are the far differences at modes
// k0 .. k0 + n_modes - 1, whose scaled outputs are written into mode slices.
struct MlpArgs {
    const float* params = nullptr;  // BF16-rounded weights in FP32 storage, packed as in fbc.h
    int H = 0;
    int off[8] = {};
    int n = 0;                      // rows (per mode)
    const float* X = nullptr;       // row mode
    float* Y = nullptr;
    const int2* far = nullptr;      // slice mode
    int k0 = 0, n_modes = 1, L = 0;
    double c = 1.0;
    float* slice = nullptr;         // [n_modes][Dy][Dx][6]
    int Dx = 0, box_x0 = 0, box_y0 = 0;
    size_t slice_floats = 0;        // Dy * Dx * 6
    int* status = nullptr;
};
bool mlp_tc_supported(int H);
cudaError_t launch_mlp_tc(const MlpArgs& a, cudaStream_t st);

// Conversions between double and float on the integer pipes (GB300's FP64
// pipe, where cvt between the two issues, runs at about 1/64 of the FP32 rate).
// double -> float, rounded to nearest (ties away from zero); magnitudes below
// 2^-126 become signed zero (no overflow for the values transformed here).
__device__ __forceinline__ float d2f_bits(long long bits) {
    const unsigned long long b = (unsigned long long)bits;
    const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
    const unsigned int sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    unsigned int r = ((unsigned int)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    r += (lo >> 28) & 1u;  // a carry out of the mantissa raises the exponent, as it should
    return __uint_as_float(sign | r);
}
__device__ __forceinline__ float d2f_int(double x) { return d2f_bits(__double_as_longlong(x)); }
// float -> double, exact; zero and FP32 subnormals become signed zero.
__device__ __forceinline__ double f2d_int(float x) {
    const unsigned int b = __float_as_uint(x);
    const unsigned int sign = b & 0x80000000u, e = (b >> 23) & 0xffu;
    if (e == 0) return __longlong_as_double((long long)((unsigned long long)sign << 32));
    const unsigned int hi = sign | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    const unsigned int lo = (b & 7u) << 29;
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}
// Record the message fbc_last_error() returns for this thread; returns code.
int report_error(int code, const char* msg);

// The FP32 line transforms run in the Stockham form up to this L (two padded buffers of 1.5 NC L FP32
// complex numbers: 110 KB at L = 2048), when the caller's arrays are 16-byte aligned; else radix-2.
constexpr int kLineStockhamMaxL = 2048;
bool line_stockham(int L, const void* a, const void* b);

// line-transform blocking: columns per CTA so that a CTA holds 2048 complex points
inline int line_cols(int L) {
    int nc = 2048 / L;
    if (nc < 2) nc = 2;
    if (nc > 64) nc = 64;
    return nc;
}

}  // namespace fbc

struct fbc_plan {
    fbc::Plan p;
};

