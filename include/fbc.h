/*
 * fbc.h -- C ABI of the GB300 (sm_103a) Green's-function pad update of the
 * flexible boundary condition (FBC) method for line-periodic dislocations.
 *
 * The operation (Sec. 1, Eq. 1; Sec. 2.3.2, Eq. 22 and Algorithm 1;
 * Sec. 3.2, Eqs. 37-38): given the forces f on the interface atoms, update
 * the displacements u of the pad atoms,
 *
 *     u(a, p) <- beta * u(a, p) + alpha * sum_{b, q} G~(x_a - x_b, (p - q) c) f(b, q),
 *
 * where a runs over the pad columns, b over the interface columns, p, q over
 * the L repeats of each column along the periodic line (spacing c, period
 * l3 = L c), and G~ is the regularised periodic Green function of Sec. 3.1,
 * Eqs. 32-36 (image sum with Richardson extrapolation).  The paper's own
 * update is alpha = -1 (or the relaxation factor of Algorithm 1), beta = 1.
 *
 * Because G~ is l3-periodic along the line, the sum over q is a circular
 * convolution.  The library evaluates it exactly by a DFT along the line:
 * forward FFT of f, an independent dense complex 3x3-block contraction per
 * wavenumber k = 0..L/2 against a table g^k(d) indexed by the in-plane
 * lattice difference d = x_a - x_b, and an inverse FFT.
 *
 * Conventions shared by every entry point
 *   - Sites are integer lattice sites x in Z^2 (one per atom column).
 *   - Force and displacement arrays are row-major [n_rhs][N][L][3] (FP64
 *     unless the name says f32), resident in DEVICE memory unless the entry
 *     point says host; the caller owns them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream are asynchronous on it, do not
 *     synchronise the host and do not allocate.
 *   - Every call returns an fbc status code; the message of the last failure
 *     on the calling thread is available from fbc_last_error().  No call
 *     exits or aborts the process.
 */
#ifndef FBC_H
#define FBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define FBC_OK 0
#define FBC_ERR_INVALID_ARG 1   /* a pointer, size or option is out of range */
#define FBC_ERR_OOM 2           /* device or host allocation failed */
#define FBC_ERR_CUDA 3          /* a CUDA runtime call or kernel launch failed */
#define FBC_ERR_NOT_TABULATED 4 /* fbc_apply before fbc_tabulate_kernel */
#define FBC_ERR_TIMEOUT 5       /* a bounded device wait gave up */
#define FBC_ERR_UNSUPPORTED 6   /* valid request this build does not implement */

/* ---- material kinds -------------------------------------------------- */
#define FBC_MATERIAL_ISOTROPIC 0 /* Kelvin's closed form (mu, nu) */
#define FBC_MATERIAL_CUBIC 1     /* Barnett's line integral (C11, C12, C44, Q) */

/* ---- contraction precisions (fbc_options.precision) ------------------ */
#define FBC_PREC_FP64 0  /* FP64 fused multiply-add throughout */
#define FBC_PREC_FP32 1  /* FP32 products and sums; k = 0 mode kept in FP64 */
#define FBC_PREC_F32X2 2 /* double-float: FP64-accurate products/sums built from FP32 pairs */
#define FBC_PREC_TF32 3   /* tensor cores (tcgen05): tf32 operands, FP32 accumulation; k = 0 in FP64 */
#define FBC_PREC_BF16X2 4 /* tensor cores: bf16 split x = h + m, 3 products, FP32 accumulation; k = 0 in FP64 */
#define FBC_PREC_BF16X3 5 /* tensor cores: bf16 split x = h + m + l, 6 products, FP32 accumulation; k = 0 in FP64 */
/* In-plane FFT form (FP64): the per-mode sum over interface columns is a 2D
 * convolution over the lattice (the kernel depends only on x_a - x_b), done
 * exactly as a circular convolution on a power-of-two grid of at least
 * 2 max|d| + 1 points per side, O(M log M) per mode instead of
 * O(N_P N_I).  Needs the grid's transformed kernel (6 reals per grid point
 * and mode, built on first use) and a workspace of at most about 1 GiB.
 * Not for batches or plans with a surrogate. */
#define FBC_PREC_FFT64 6
/* The in-plane FFT form with FP32 transforms and kernel for the modes k >= 1
 * and FP32 line transforms; the logarithmic k = 0 mode stays on the FP64
 * grid transforms (as the other FP32 forms keep it FP64-accurate). */
#define FBC_PREC_FFT32 7
/* Tensor cores, FP64-accurate (Ozaki's error-free splitting of the dot
 * product; Sec. 3.2, Eqs. 37-38 as the other forms), for plans with several
 * right-hand sides: every table entry and force value, scaled by a power of
 * two (one per pad tile and interface tile pair; one per force column and
 * mode), is cut into six fixed-point bf16 slices of 8 bits.  The 26 slice
 * products with i + j <= 8 are summed in FP32 tensor memory -- exactly for the
 * diagonals i + j = 2 .. 5, one accumulator each, the diagonals 6 .. 8 in a
 * shared one -- over groups of 64 interface columns, which are combined in
 * double-float.  Per term the error is about 2^-47 of the largest operand
 * product of the tile pair; measured 2e-13 relative L2 against the FP64
 * oracle at 8000 x 12000 columns, L = 1024.  Runs 32 right-hand sides per CTA
 * (fewer waste the rest of the group).  Needs the double-float table, FP64
 * line transforms and a sliced force operand of 36 KB per (mode, group of 32
 * rhs, stage of 16 interface columns); k = 0 in double-float.  Force and
 * table magnitudes must lie within about 2^-118 .. 2^118.  Not for batches or
 * plans with a surrogate. */
#define FBC_PREC_BF16X6 8

/* ---- plan flags (fbc_options.flags) ----------------------------------- */
#define FBC_PLAN_HOST_ONLY 1 /* validate and lay out on the host only: no device memory,
                                tabulate/apply are refused; for inspecting the layout */
/* Tensor-core forms: the FP32 accumulation in tensor memory truncates at every
 * step, so by default the interface sum is split into groups of 1024 interface
 * columns whose partial sums are added with round-to-nearest FP32 adds.  This
 * flag keeps the whole sum in one group: about 15 % faster at 8000 interface
 * columns, with an accumulation error about 8x larger (1.1e-4 instead of
 * 1.2e-5 for BF16X2 there).  Plans with at most 1024 interface columns are
 * not affected. */
#define FBC_PLAN_TC_FAST_ACCUMULATE 2
/* Interface and pad sites may coincide, as in the paper (Lambda^{i+} inside
 * Lambda^p, self-terms d = 0).  The continuum kernel is singular at d = 0,
 * so those table entries are zero until fbc_plan_lattice_near_field replaces
 * them (it always covers d = 0); applies are refused until then, and again
 * after a new tabulation. */
#define FBC_PLAN_SELF_TERMS 4

/* ---- fbc_apply flags ------------------------------------------------- */
#define FBC_APPLY_PROJECT_NEUTRAL 1u /* remove the net interface force first */
#define FBC_APPLY_ZERO_MEAN_U 2u     /* set the mean pad displacement to zero after (Eq. 23) */
#define FBC_APPLY_NO_GRAPH 4u        /* fbc_batch_apply only: launch directly instead of replaying a graph */

/* Column geometry (Sec. 2.1: line-periodic slab of a Bravais lattice).
 * The interface columns are the force sources (the paper's Lambda^{i+}),
 * the pad columns the targets (Lambda^p).  The two site lists are copied at
 * plan creation; they must be disjoint and free of duplicates. */
typedef struct fbc_geometry {
    int32_t n_i;          /* number of interface columns, >= 1 */
    int32_t n_p;          /* number of pad columns, >= 1 */
    int32_t L;            /* repeats along the line: a power of two in [2, 4096] */
    double c;             /* spacing along the line, > 0 (period l3 = L c) */
    const int32_t* xy_i;  /* HOST [n_i][2] integer in-plane sites */
    const int32_t* xy_p;  /* HOST [n_p][2] integer in-plane sites */
} fbc_geometry;

/* Elastic medium of the continuum Green function (Sec. 3.1, Eq. 33).
 * Q is the row-major rotation from the computational frame to the crystal
 * frame (r_crystal = Q r); the Green function in the computational frame is
 * Q^T G(Q r) Q (App. B).  Only media symmetric under the mirror x3 -> -x3
 * (isotropic media, or a cubic crystal with a cube axis along the line) are
 * accepted; other rotations return FBC_ERR_UNSUPPORTED. */
typedef struct fbc_material {
    int32_t kind;             /* FBC_MATERIAL_* */
    double mu, nu;            /* isotropic: shear modulus > 0, -1 < nu < 0.5 */
    double C11, C12, C44;     /* cubic constants, crystal frame (stable medium) */
    double Q[9];              /* rotation; all zero is read as the identity */
} fbc_material;

/* Plan options; fbc_default_options() fills the defaults. */
typedef struct fbc_options {
    int32_t precision;  /* FBC_PREC_*, default FBC_PREC_FP64 */
    int32_t rich_n;     /* Richardson n (Eq. 36), default 4 */
    int32_t rich_N;     /* Richardson order N (Eq. 36), default 6; n_img = n + N */
    int32_t quad;       /* Barnett trapezoid nodes on [0, pi), default 64 */
    int32_t max_rhs;    /* largest n_rhs fbc_apply will accept, default 1 */
    int32_t flags;      /* FBC_PLAN_* bits, default 0 */
} fbc_options;

typedef struct fbc_plan fbc_plan;

/* Read-only description of a plan (sizes and the layout the kernels use). */
typedef struct fbc_plan_info {
    int32_t n_i, n_p, L, K;     /* K = L/2 + 1 wavenumbers */
    int32_t max_rhs, precision;
    int32_t tile_a, tile_b;     /* pad / interface columns per tile */
    int32_t n_tiles_a, n_tiles_b;
    int32_t box_x0, box_y0;     /* in-plane origin of the difference table */
    int32_t box_nx, box_ny;     /* its extent (columns of d_x, rows of d_y) */
    int32_t sub_w, sub_h;       /* largest per-tile-pair sub-box */
    int32_t n_used_d;           /* differences that occur between the two sets */
    int32_t tabulated;          /* 1 after fbc_tabulate_kernel */
    double pair_modes_per_rhs;  /* n_p * n_i * K */
    size_t table_bytes;         /* FP64 mode table */
    size_t workspace_bytes;     /* everything else the plan owns on the device */
    size_t surrogate_bytes;     /* buffers of an attached surrogate (slice, near copy, lists, activations) */
    int32_t surrogate_attached; /* 1 while a surrogate is attached */
    int32_t n_far_d;            /* used differences the surrogate serves (|d| >= r_min) */
    int32_t surrogate_chunk;    /* modes per streamed chunk (one network, near-copy and contraction launch each) */
    int32_t reserved;
    int32_t fft_mx, fft_my;     /* in-plane FFT form: grid (0 until built) */
    int32_t fft_rows_i, fft_rows_p; /* grid rows holding interface / pad sites */
    int32_t fft_chunk_items;    /* (rhs, mode) items per workspace chunk: 3 launches each */
    int32_t reserved2;
} fbc_plan_info;

/* Defaults listed in fbc_options. */
void fbc_default_options(fbc_options* opt);

/* The setup of the pad update, done once and reused by every later apply
 * (Sec. 3.2: the Green matrix is built once per geometry and only applied
 * afterwards).  The geometry is the line-periodic slab of Sec. 2.1 (columns
 * of L atoms at in-plane lattice sites, the interface set Lambda^{i+} and the
 * pad Lambda^p), the medium that of the Green function of Sec. 3.1, Eq. 33.
 * Validate the geometry and medium, sort the columns into spatially compact
 * tiles and allocate every device buffer the plan will need (tables and the
 * workspace for max_rhs right-hand sides).  Rejects: non-power-of-two L,
 * coincident interface/pad sites (d = 0, where the continuum kernel is
 * singular), duplicate sites, unsupported media.  On success *out owns the
 * plan; on failure *out is NULL.  Synchronous; uses the current device. */
int fbc_plan_create(const fbc_geometry* geom, const fbc_material* mat, const fbc_options* opt,
                    fbc_plan** out);

/* Tabulate the periodic kernel and its per-mode table (Sec. 3.1, Eqs. 32-36,
 * then a DFT along the line): for every in-plane difference d that occurs and
 * every wavenumber k, g^k(d) = sum_s G~(d, s c) exp(-2 pi i k s / L), stored as
 * six reals [Re g11, Re g12, Re g22, Re g33, Im g13, Im g23] (the other
 * parts vanish by the mirror symmetry).  Runs once per plan; the table is
 * reused by every apply (Sec. 3.2: the setup is reused across runs).
 * Asynchronous on `stream`, except that for the in-plane FFT forms the first
 * call also builds the grid (host structures and device buffers: synchronous,
 * allocates) before it queues the grid transform of the table. */
int fbc_tabulate_kernel(fbc_plan* plan, void* stream);

/* The pad update (see the top of this file) for n_rhs right-hand sides:
 *   f: DEVICE const double [n_rhs][n_i][L][3], interface forces (original order);
 *   u: DEVICE double [n_rhs][n_p][L][3], pad displacements, updated in place
 *      (read only when beta != 0);
 *   flags: FBC_APPLY_PROJECT_NEUTRAL removes the per-component mean of f over
 *      all n_i * L interface atoms (per right-hand side) before the update;
 *      FBC_APPLY_ZERO_MEAN_U subtracts the per-component mean of the updated u
 *      over all n_p * L pad atoms (Sec. 2.3.2, Eq. 23).
 * 1 <= n_rhs <= max_rhs.  f and u must not overlap.  The contraction runs in
 * the plan's precision.  Asynchronous on `stream`; concurrent applies of one
 * plan on different streams race on its workspace. */
int fbc_apply(fbc_plan* plan, const double* f, double* u, int32_t n_rhs, double alpha, double beta,
              uint32_t flags, void* stream);

/* Relaxed pad update of the FBC iteration (Algorithm 1 with the residual-based
 * relaxation of Sec. 2.3.3, Algorithm 2), per right-hand side r:
 *   alpha = -alpha_io[r] <f_old, f_new - f_old> / ||f_new - f_old||^2   (f_old given;
 *           kept as alpha_io[r] if f_new == f_old),
 *   alpha = 1 if it is negative,
 *   alpha = du_max / ||G f_new||_inf if du_max > 0 and ||alpha G f_new||_inf > du_max,
 *   u <- u - alpha G f_new, then the optional zero mean (FBC_APPLY_ZERO_MEAN_U),
 * and alpha_io[r] <- alpha.  The inner products run over all n_i * L interface
 * atoms and components of the raw inputs; the maximum over all n_p * L pad atoms
 * and components of G f_new (after the optional neutral projection of f_new, as
 * in fbc_apply).  f_old = NULL skips the first two steps (alpha_io is used as
 * given, as in the iterations before the relaxation starts).
 *   f_new, f_old: DEVICE double [n_rhs][n_i][L][3]; u: DEVICE double
 *   [n_rhs][n_p][L][3] (updated in place); alpha_io: DEVICE double [n_rhs].
 * Asynchronous on `stream`; no allocation and no host synchronisation (alpha is
 * computed on the device).  The plan's contracted modes are transformed twice
 * (once for the maximum, once for the update) when du_max > 0. */
int fbc_apply_relaxed(fbc_plan* plan, const double* f_new, const double* f_old, double* u, int32_t n_rhs,
                      double* alpha_io, double du_max, uint32_t flags, void* stream);

/* Same as fbc_apply with f and u in HOST memory (pinned memory makes the
 * copies asynchronous): copies f (and u when beta != 0) to the plan's device
 * staging buffers, applies, copies u back and synchronises `stream`.  The
 * right-hand sides go through in at most 8 chunks of at least 4 (for the
 * tensor-core forms: of whole right-hand-side groups, 32 for FBC_PREC_BF16X6
 * and up to 64 for the others): each chunk is copied in on a stream of the
 * plan, applied on `stream`, and copied out on a second stream of the plan,
 * so the copies of one chunk overlap the applies of the others.  Each
 * right-hand side is computed as in one fbc_apply of all of them (for the
 * CUDA-core forms and FBC_PREC_BF16X6 with the same bits).  The first call allocates the staging buffers and creates
 * the two streams. */
int fbc_apply_host(fbc_plan* plan, const double* f_host, double* u_host, int32_t n_rhs, double alpha,
                   double beta, uint32_t flags, void* stream);

/* Switch the contraction precision of an existing plan.  Builds the
 * precision's derived table from the FP64 table on first use (allocates;
 * call outside stream capture): the FP32 or double-float table, or for the
 * in-plane FFT forms the grid and its transformed kernel (K x Mx x My x 6
 * reals in FP64, plus an FP32 copy for FBC_PREC_FFT32).  Synchronous. */
int fbc_plan_set_precision(fbc_plan* plan, int32_t precision);

/* Bound of the pipeline waits of the tensor-core contraction (the hand-offs
 * of shared-memory stages between its warps), in polls of the barrier:
 * 1 <= polls <= 2^24, or 0 for the default 2^24.  A wait that runs out stops
 * the contraction's work; the next fbc_plan_sync_status then returns
 * FBC_ERR_TIMEOUT (the results of that apply are not valid).  The waits for
 * the kernel's own copies and products in flight, before it frees its tensor
 * memory and exits, always keep the default bound.  Meant for tests of the
 * timeout path; host only, takes effect at the next apply. */
int fbc_plan_set_wait_limit(fbc_plan* plan, int32_t polls);

/* Stage timing for profiling.  While enabled, every fbc_apply records CUDA
 * events on its stream before the forward transform, after it, after the
 * per-mode contraction and after the inverse transform.  Synchronous. */
int fbc_plan_set_timing(fbc_plan* plan, int32_t enable);

/* Durations of the last timed apply, in milliseconds: ms[0] forward
 * transform (and projection), ms[1] contraction, ms[2] inverse transform
 * (and zero mean).  Waits for that apply's events. */
int fbc_plan_stage_times(fbc_plan* plan, float* ms);

/* Fill *info.  Host only. */
int fbc_plan_info_get(const fbc_plan* plan, fbc_plan_info* info);

/* Host copy of the tile-sorted layout the kernels use (host only, works on a
 * FBC_PLAN_HOST_ONLY plan).  With NIpad = n_tiles_b * tile_b and
 * NPpad = n_tiles_a * tile_a from fbc_plan_info:
 *   perm_i: [NIpad] original interface column of each sorted slot, -1 = padding;
 *   perm_p: [NPpad] same for the pad columns;
 *   xy_i:   [NIpad][2] site of each sorted interface slot (padding repeats
 *           the first site of its tile);
 *   xy_p:   [NPpad][2] same for the pad slots.
 * Any output pointer may be NULL. */
int fbc_plan_layout(const fbc_plan* plan, int32_t* perm_i, int32_t* perm_p, int32_t* xy_i, int32_t* xy_p);

/* Lattice Green function near field (App.: the lattice Green function up to
 * a cut-off, the continuum one beyond, joined by a blending constant).  For
 * every difference d of the plan's table with |d| <= r_cut, the mode entries
 * g^k(d) are replaced by the lattice Green function of the harmonic block
 * stencil K [27][3][3] (HOST, the layout of fbc_stencil_create):
 *     g^k(d) = (2 pi)^-2 int D(theta_x, theta_y, 2 pi k / L)^-1 exp(i theta . d),
 *     D(theta) = sum_n K(n) exp(-i theta . n),
 * evaluated by the trapezoid rule on an n x n grid of the zone (n = n_zone
 * rounded up to 2^a 3^b 5^c; 16 <= n_zone <= 2048), i.e. by 2D FFTs.  The
 * modes k >= 1 are used as computed.  The k = 0 mode (symbol singular at
 * theta = 0, left out) is defined up to a constant: it is shifted by
 * C = g_lat^0(d_ref) - g^0(d_ref), d_ref = (ref_dx, ref_dy) a difference of
 * the plan's table with |d_ref| > r_cut (the paper's r', far enough that C
 * hardly depends on it); d_ref = (0, 0) leaves the k = 0 mode as computed
 * (the zero-mean function; for a table that is lattice throughout).  The
 * stencil must satisfy
 * K(-n) = K(n) and the mirror symmetry along the line (FBC_ERR_UNSUPPORTED
 * otherwise); the grid must exceed twice the largest |d_x|, |d_y| involved.
 * Call after fbc_tabulate_kernel, and again after a later tabulation; the
 * precision's derived table is rebuilt.  Synchronous; allocates temporary
 * device memory (about n^2 x 144 B per mode, in chunks of at most 512 MB). */
int fbc_plan_lattice_near_field(fbc_plan* plan, const double* K, double r_cut, int32_t ref_dx, int32_t ref_dy,
                                int32_t n_zone);

/* Copy rows of the FP64 mode table to the host (synchronous):
 *   d:   HOST [nd][2] in-plane differences (each must lie in the table box);
 *   out: HOST double [nd][K][6] in the six-real layout of fbc_tabulate_kernel. */
int fbc_get_mode_table(const fbc_plan* plan, const int32_t* d, int32_t nd, double* out);

/* Wait for the plan's work on `stream` and report a device-side error word
 * (FBC_ERR_TIMEOUT if a bounded wait gave up).  Clears the word. */
int fbc_plan_sync_status(fbc_plan* plan, void* stream);

/* Release every resource of the plan (synchronises the device first).
 * NULL is ignored. */
void fbc_destroy(fbc_plan* plan);

/* Message of the last failing call on this thread ("" if none).  The
 * string is owned by the library and valid until the next call. */
const char* fbc_last_error(void);

/* Library version string. */
const char* fbc_version(void);

/* ---- batches of plans ------------------------------------------------
 * Many independent FBC instances (uneven sizes, each with its own right-hand
 * sides) updated together -- the pad update of Eqs. 1, 22, 37-38 for each
 * instance -- by one fixed sequence of launches: batched line transforms and
 * ONE persistent contraction launch that drains a cost-sorted tile queue over
 * all instances (no CTA ever waits for another), captured into a CUDA graph
 * on first use and replayed. */
typedef struct fbc_batch fbc_batch;

typedef struct fbc_batch_info {
    int32_t n_plans, precision;
    int32_t n_contract_items;   /* (instance, mode, pad tile, rhs block) work items */
    int32_t grid;               /* persistent contraction CTAs */
    int32_t occupancy;          /* resident contraction CTAs per SM */
    int32_t lpt_order;          /* 1: longest-first queue, 0: instance-major */
    int32_t kernel_launches;    /* launches per apply (with both flags) */
    size_t smem_contract;       /* dynamic shared memory of the contraction CTAs */
    double pair_modes;          /* sum over instances of n_p n_i K n_rhs */
    int32_t rhs_per_cta;        /* right-hand sides per contraction work item (tensor forms: the tuned group) */
    int32_t launch_form;        /* tensor forms: 0 one persistent launch over all items, 1 per-instance launches */
} fbc_batch_info;

/* Bind n_plans tabulated plans (same precision, each at most once) to their
 * DEVICE buffers: f[i] [n_rhs[i]][n_i][L][3], u[i] [n_rhs[i]][n_p][L][3].
 * The buffers are fixed for the batch's lifetime (the graph refers to them).
 * Precisions: FP64, FP32, double-float and the tensor-core forms (TF32,
 * BF16X2, BF16X3: the modes k >= 1 of every instance run in one persistent
 * tensor-core launch, k = 0 in double-float; a timeout of that launch is
 * reported through the first plan's status word, fbc_plan_sync_status).  Not
 * the in-plane FFT forms.  Allocates the work lists; synchronous. */
int fbc_batch_create(fbc_plan* const* plans, int32_t n_plans, const double* const* f, double* const* u,
                     const int32_t* n_rhs, fbc_batch** out);

/* u_i <- beta u_i + alpha G_i f_i for every instance (flags as fbc_apply, plus
 * FBC_APPLY_NO_GRAPH).  The first call with a new (alpha, beta, flags)
 * captures the launch sequence into a CUDA graph (on an internal stream);
 * later calls replay it on `stream`.  Asynchronous; do not run two applies of
 * one batch, or of batches sharing a plan, concurrently. */
int fbc_batch_apply(fbc_batch* batch, double alpha, double beta, uint32_t flags, void* stream);

/* Time the contraction for each candidate configuration and keep the fastest
 * (synchronous; reallocates the queue): both queue orders (longest first,
 * instance-major) and, for the CUDA-core forms, a few persistent grid sizes;
 * for the tensor-core forms the launch form (one persistent launch over the
 * items of all instances, or each instance's own launches inside the graph)
 * and the queue's rhs group (right-hand sides per work item, i.e. the N = 2
 * rhs of the tensor-core tile: the plans' largest, then halves down to 8).
 * No candidate changes the results.  *best_ms (may be NULL) receives the
 * chosen configuration's contraction time. */
int fbc_batch_autotune(fbc_batch* batch, void* stream, double* best_ms);

int fbc_batch_info_get(const fbc_batch* batch, fbc_batch_info* info);

/* Release the batch (not its plans).  NULL is ignored. */
void fbc_batch_destroy(fbc_batch* batch);

/* Allocation-free zero-mean step.  The paper has no counterpart of this
 * call: it exists for callers that cannot call cudaMalloc where they need
 * it -- an atomistic engine that owns the whole device through its own
 * memory pool, or a relaxation loop that must not take the allocator's
 * device-wide lock.
 *   u: DEVICE double [n_rhs][n_p][L][3]; for every right-hand side and
 *      component the mean over all n_p * L pad atoms is subtracted in place
 *      (the same result as the FBC_APPLY_ZERO_MEAN_U step of fbc_apply).
 * 1 <= n_rhs <= 64; larger n_rhs returns FBC_ERR_INVALID_ARG.  Needs no
 * plan.  The reduction scratch is a fixed 384 KiB array inside the library
 * that every GPU loading the library keeps until the process exits; all
 * calls share it, so calls that overlap on the GPU race.  The first call on
 * a device looks up the array's device address (make it before any stream
 * capture); calls outside a capture look it up again, so after a
 * cudaDeviceReset make one call outside a capture first.  Asynchronous on
 * `stream`; allocates nothing. */
int fbc_zero_mean_static(double* u, int32_t n_rhs, int32_t n_p, int32_t L, void* stream);

/* ---------------------------------------------------------------------------
 * Incompatibility force (Sec. 2.3.2, Eq. 21; Algorithm 1, the step between
 * the atomistic solve and the pad update): the harmonic operator L_h,
 * restricted to the rows of the interface columns Lambda^{i+}, applied to
 * the displacements of the sites around them -- the relaxed atoms with their
 * new displacements u_{k+1}, the continuum nodes with the previous ones u_k:
 *     f_in = L_h^{i+|i}[u_{k+1}] + L_h^{i+|i++}[u_k].
 * L_h is a local block stencil on the line-periodic lattice,
 *     L_h[u](x, q) = sum_{n in {-1,0,1}^3} K(n) u(x + (n_x, n_y), (q + n_z) mod L),
 * K [27][3][3] row-major with offset index (n_x+1)*9 + (n_y+1)*3 + (n_z+1);
 * an all-zero block is skipped.  The result feeds fbc_apply_relaxed as its
 * f_new (and, one iteration later, as its f_old).
 * ------------------------------------------------------------------------- */
typedef struct fbc_stencil fbc_stencil;

#define FBC_STENCIL_MAX_SOURCES 4

/* Force constants of a synthetic harmonic model (the paper's EAM force
 * constants are not available): a simple lattice with in-plane spacing 1 and
 * plane spacing c, central springs of stiffness k1 to the 6 neighbours with
 * |n|_1 = 1 and k2 to the 12 with |n|_1 = 2.  For a spring of stiffness k
 * along v = (n_x, n_y, c n_z): K(n) = -k v v^T / |v|^2, and
 * K(0) = -sum_{n != 0} K(n) (a rigid translation gives no force).  For
 * c = 1 the long-wave limit is the cubic medium C11 = k1 + 2 k2,
 * C12 = C44 = k2.  Host only: writes K [27][3][3]. */
int fbc_spring_constants(double k1, double k2, double c, double* K);

/* Build the stencil for the interface columns xy_i [n_i][2] (the rows) and
 * n_src source site sets xy_src[s] [n_site[s]][2] (host arrays; ownership
 * stays with the caller).  Every in-plane neighbour of an interface site
 * that a non-zero block reaches, the site itself included, must be in
 * exactly one source set: a missing site, or a site in two sets, returns
 * FBC_ERR_INVALID_ARG before anything is allocated.  L >= 1 planes.
 * Uploads the neighbour table (36 B per interface column) and K.
 * Synchronous. */
int fbc_stencil_create(int32_t n_i, const int32_t* xy_i, int32_t n_src, const int32_t* const* xy_src,
                       const int32_t* n_site, int32_t L, const double* K, fbc_stencil** out);

/* f_in[r][a][q][:] = L_h[u](x_a, q) for every right-hand side r, interface
 * column a and plane q, with u taken from the source set holding each site:
 *   u_src: HOST array of n_src DEVICE pointers, u_src[s] double
 *          [n_rhs][n_site[s]][L][3] (NULL allowed for an empty set);
 *   f_in:  DEVICE double [n_rhs][n_i][L][3], overwritten; must not alias
 *          any u_src[s].
 * FP64 fused multiply-adds in a fixed order.  Asynchronous on `stream`;
 * allocates nothing. */
int fbc_incompat_force(const fbc_stencil* st, const double* const* u_src, double* f_in, int32_t n_rhs,
                       void* stream);

/* Free the stencil's device buffers (NULL is a no-op). */
int fbc_stencil_destroy(fbc_stencil* st);

/* ---------------------------------------------------------------------------
 * Learned surrogate of the mode table (an extension; the paper tabulates the
 * kernel exactly and has no learned model).  For a difference d != 0 and a
 * mode k >= 1 a multilayer perceptron 4 -> H -> H -> H -> 6 with SiLU
 * activations maps the features
 *     x = (ln(q r) / 4, d_x / r, d_y / r, ln(r) / 5),  r = |d|,  q = 2 pi k / (L c)
 * to the six reals [A11, A12, A22, A33, B13, B23] of the mode table (the
 * layout fbc_get_mode_table returns), divided by the scale
 *     s(q, r) = exp(-q r) / (c sqrt(1 + q r)),
 * the decay of the modified Bessel functions K_0, K_1 that the line sum of
 * the Green function (Eqs. 32-36) becomes for k >= 1.  Entries with
 * q r > 16 (below exp(-16) of the entry at q r -> 0, and below the FP64
 * table's own roundoff after Richardson extrapolation) are served as zero;
 * training samples only q r <= 16.  Parameters are FP32 master weights (He
 * initialisation from `seed`), trained with Adam on samples of the plan's
 * exact FP64 table; inference uses the weights rounded to BF16 with FP32
 * accumulation (a fused tensor-core kernel for H in {32, 64, 96, 128}).
 * Layout of the parameter vector: W1 [4][H], b1 [H], W2 [H][H], b2 [H],
 * W3 [H][H], b3 [H], W4 [H][6], b4 [6] (row = input).  The surrogate object
 * owns its device buffers.
 * ------------------------------------------------------------------------- */
typedef struct fbc_surrogate fbc_surrogate;

/* Create a surrogate of hidden width H (multiple of 8 in [8, 1024]). */
int fbc_surrogate_create(int32_t width, uint64_t seed, fbc_surrogate** out);

/* Number of parameters (4H + H + 2(H^2 + H) + 6H + 6); 0 for NULL. */
int fbc_surrogate_n_params(const fbc_surrogate* s);

/* Copy the FP32 master parameters: host_in (may be NULL) is written to the
 * device first, then the device copy is read into host_out (may be NULL). */
int fbc_surrogate_params(fbc_surrogate* s, float* host_out, const float* host_in);

/* Network output y[n][6] = MLP(x[n][4]) (scaled units, no s(q, r)).
 * x, y: DEVICE float.  bf16_weights != 0 uses the BF16-rounded weights (and,
 * for the widths it takes, the fused tensor-core kernel, whose waits are
 * bounded: a timeout is reported by fbc_surrogate_sync_status).
 * Asynchronous on `stream`. */
int fbc_surrogate_forward(fbc_surrogate* s, const float* x, float* y, int32_t n, int32_t bf16_weights, void* stream);

/* Wait for `stream` and report a timeout of the fused inference kernel
 * (FBC_ERR_TIMEOUT, after which the word is cleared). */
int fbc_surrogate_sync_status(fbc_surrogate* s, void* stream);

/* Mean squared error  loss = sum_i sum_j (y_ij - t_ij)^2 / (6 n)  over the
 * FP32 weights and its gradient.  x[n][4], t[n][6]: DEVICE float.  loss
 * (host double, may be NULL) and host_grad (host float[n_params], may be
 * NULL) are written after the stream synchronises. */
int fbc_surrogate_loss_grad(fbc_surrogate* s, const float* x, const float* t, int32_t n, double* loss,
                            float* host_grad, void* stream);

/* Train on n_samples pairs (d, k) drawn (seeded) from the plan's differences
 * with |d| >= r_min -- d uniform, k log-uniform over the modes 1 <= k < K
 * with q r <= 16 -- with targets from the exact FP64 table divided by
 * s(q, r): `epochs` passes of Adam (beta 0.9, 0.999) over batches
 * of `batch`, learning rate lr decayed by a half cosine over the epochs.
 * final_loss (may be NULL) receives the last batch's loss.  The plan must be
 * tabulated.  Blocks until done. */
int fbc_surrogate_train(fbc_surrogate* s, const fbc_plan* plan, int32_t n_samples, double r_min, int32_t epochs,
                        int32_t batch, double lr, uint64_t seed, void* stream, double* final_loss);

/* Surrogate mode-table entries for n pairs: d[n][2] (host int32, d != 0),
 * k[n] (host int32, 1 <= k < K); out[n][6] (host double) in the layout of
 * fbc_get_mode_table, BF16 weights.  Blocks until done. */
int fbc_surrogate_eval_table(fbc_surrogate* s, const fbc_plan* plan, const int32_t* d, const int32_t* k, int32_t n,
                             double* out);

/* Attach a trained surrogate (width 32, 64, 96 or 128) to a plan whose
 * precision is FBC_PREC_FP32 or a tensor-core form.  fbc_apply then builds,
 * for a chunk of modes k >= 1 at a time (as many as fit in about 48 MB), FP32
 * mode slices in device memory -- the network for |d| >= r_min, a compact
 * FP32 copy of the exact table for the near differences -- and contracts with
 * them in one launch per chunk; mode k = 0 stays exact.  A timeout of the
 * network kernel is reported through the plan's status word.  release_tables != 0 frees the plan's K-slice
 * tables (FP64 and derived), keeping only the near copy and the k = 0 slice:
 * the plan can then neither be re-tabulated nor switch precision, and
 * fbc_get_mode_table fails.  s == NULL detaches (refused once tables were
 * released).  The plan keeps a pointer to s: s must outlive the plan or be
 * detached first; later training of s takes effect at the next attach. */
int fbc_plan_attach_surrogate(fbc_plan* plan, fbc_surrogate* s, double r_min, int32_t release_tables);

/* Release the surrogate.  NULL is ignored. */
void fbc_surrogate_destroy(fbc_surrogate* s);


/* Measured rate of fused multiply-adds on this GPU, for the rooflines of the CUDA-core forms:
 * FP32 (fp64 = 0) or FP64 (fp64 = 1), 2 flops per FMA.  8 CTAs of 256 threads per SM run 8
 * independent chains per thread; the second of two launches is timed with events on `stream`.
 * *tflops receives TFLOP/s.  Blocks until done; allocates a small buffer. */
int fbc_measure_fma_peak(int32_t fp64, double* tflops, void* stream);

/* ---------------------------------------------------------------------------
 * H-matrix form of the pad update (Sec. 3.2; App., the construction of the
 * H-matrix approximation of the Green matrix): the comparison form.  The
 * Green matrix G~^{p|i+} has 3 x 3 blocks G~(x_a - x_b, (p - q) c) for pad atoms
 * (a, p) and interface atoms (b, q).  It is approximated by
 *   Step 1: cluster trees of each atom set by geometric bisection: split at
 *           the midpoint of the bounding box's longest side until at most
 *           b_min atoms;
 *   Step 2: the admissible partition: t x s is low rank when
 *           min(diam t, diam s') <= gamma dist(t, s') for s' in {s, s+, s-},
 *           where s+- are the same cluster one period L c up and down, diam
 *           is the bounding-box diagonal and dist the centroid distance;
 *           inadmissible pairs of leaves are dense;
 *   Step 3: adaptive cross approximation with partial pivoting on atoms
 *           (3 x 3 pivots), stopping after three consecutive steps whose
 *           terms have Frobenius norm <= eps times the approximation's.
 * The entries come from the plan's periodic kernel (Sec. 3.1, Eqs. 32-36) in
 * real space, the same kernel that the per-mode forms transform.  The build
 * runs on the device in FP32 (residuals, terms) with FP64 norms; the factors
 * are stored in FP32.  The paper's settings are eps = 1e-5, gamma = 2,
 * b_min = 20.
 * ------------------------------------------------------------------------- */
typedef struct fbc_hmat fbc_hmat;

typedef struct {
    double eps;            /* ACA tolerance, 1e-6 <= eps < 1 (paper: 1e-5) */
    double gamma;          /* admissibility constant, > 0 (paper: 2) */
    int32_t b_min;         /* leaf size of the cluster trees in atoms, 1..64 (paper: 20) */
    int32_t max_rank;      /* terms per block at most: 0 = 6141 (the build's limit), else 1..6141 */
    int64_t scratch_bytes; /* device scratch per build wave: 0 = 40 % of the free memory */
} fbc_hmat_options;

typedef struct {
    int64_t n_rows, n_cols;      /* 3 n_p L and 3 n_i L */
    int64_t n_lowrank, n_dense;  /* blocks of the partition */
    int64_t rank_sum;            /* sum of the low-rank blocks' ranks (terms) */
    int32_t rank_max;            /* the largest rank */
    int32_t n_capped;            /* blocks that stopped at max_rank before the rule held */
    int64_t factor_bytes;        /* FP32 factors U, V of the low-rank blocks */
    int64_t dense_bytes;         /* FP32 dense blocks */
    int32_t n_row_leaves, n_col_leaves;
    int32_t n_waves;             /* build waves (groups of blocks that share the scratch) */
    int32_t reserved;
    double build_ms;             /* wall time of fbc_hmat_create */
} fbc_hmat_info;

/* Steps 1 and 2 on the host only (no device use): the partition for the
 * column sites xy_i [n_i][2], xy_p [n_p][2] (host int32) with L repeats of
 * spacing c.  *n_blocks receives the number of blocks.  blocks (host int64
 * [cap][5], may be NULL) receives the blocks sorted by (row start, row count,
 * col start, col count): (row start, row count, col start, col count,
 * low rank) in atoms of cluster order, when cap >= *n_blocks
 * (FBC_ERR_INVALID_ARG otherwise).  perm_p [n_p L], perm_i [n_i L] (host
 * int64, may be NULL) receive the atom id (column * L + repeat) at each
 * cluster-order position. */
int fbc_hmat_partition(const int32_t* xy_i, int32_t n_i, const int32_t* xy_p, int32_t n_p, int32_t L, double c,
                       double gamma, int32_t b_min, int64_t* n_blocks, int64_t* blocks, int64_t cap, int64_t* perm_p,
                       int64_t* perm_i);

/* Build the H-matrix of a plan's Green matrix (the plan's geometry, medium and
 * Richardson order; its precision is not used).  Plans with interface sites
 * inside the pad (FBC_PLAN_SELF_TERMS) or a lattice near field are refused
 * (FBC_ERR_UNSUPPORTED): their kernel is not the periodic continuum one.
 * Blocks until done; allocates.  opt == NULL takes the paper's settings. */
int fbc_hmat_create(fbc_plan* plan, const fbc_hmat_options* opt, void* stream, fbc_hmat** out);

/* u <- beta u + alpha G_H f' with f' = f, or f minus its per-component mean
 * over all n_i L interface atoms (FBC_APPLY_PROJECT_NEUTRAL), then the optional
 * zero mean of u (FBC_APPLY_ZERO_MEAN_U).  f: DEVICE const double
 * [n_rhs][n_i][L][3]; u: DEVICE double [n_rhs][n_p][L][3] (read only when
 * beta != 0); n_rhs >= 1, applied four at a time.  Asynchronous on `stream`,
 * deterministic; concurrent applies of one H-matrix race on its workspace. */
int fbc_hmat_apply(fbc_hmat* h, const double* f, double* u, int32_t n_rhs, double alpha, double beta, uint32_t flags,
                   void* stream);

/* Sizes, ranks and build time. */
int fbc_hmat_get_info(const fbc_hmat* h, fbc_hmat_info* info);

/* The partition as in fbc_hmat_partition and each block's rank (ranks
 * [cap], host int32; 0 for a dense block); either may be NULL. */
int fbc_hmat_blocks(const fbc_hmat* h, int64_t* blocks, int32_t* ranks, int64_t cap);

/* Free the H-matrix (NULL is ignored). */
void fbc_hmat_destroy(fbc_hmat* h);

#ifdef __cplusplus
}
#endif
#endif /* FBC_H */
