/*
 * Plain FP64 CPU oracle for the Green's-function pad update of the flexible
 * boundary condition (FBC) method for line-periodic dislocations.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * it exists so that tests, the smoke check and the CPU baseline of the
 * benchmark have an obviously correct reference to compare the CUDA path with.
 * It shares no code, header or table with the CUDA library.
 *
 * What it computes, step by step, in the paper's notation:
 *   1. the continuum Green function G(r) of the infinite medium
 *      (Sec. 3.1, Eq. 33: G(r) = F(r_hat) / |r|) -- Kelvin's closed form for
 *      an isotropic medium, Barnett's line integral over the unit circle
 *      perpendicular to r for an anisotropic one;
 *   2. the partial sums of the regularised image sum (Sec. 3.1, Eqs. 32, 35)
 *         G_n(r) = sum_{i=-n..n} [ G(r1, r2, r3 + i l3) - G(0, 0, i l3) ],
 *      where the subtraction is skipped for i = 0 (it is singular for a
 *      continuum kernel and only shifts G by a constant);
 *   3. Richardson's extrapolation of those partial sums (Sec. 3.1, Eq. 36)
 *         Q0 = sum_{i=0..N} G_{n+i} (n+i)^N (-1)^{i+N} / (i! (N-i)!),
 *      accumulated in double-double;
 *   4. the tabulated periodic kernel on the line lattice: for repeat offset
 *      s in [0, L) the image sum is evaluated at the centred representative
 *      s' in (-L/2, L/2] (s' = s or s - L); at s = L/2 the two
 *      representatives +L/2 and -L/2 are averaged so that the table is
 *      exactly L-periodic and mirror-symmetric;
 *   5. the real-space pad update (Sec. 1, Eq. 1; Sec. 3.2, Eqs. 37-38)
 *         u(a, p) = sum_{b, q} G~(x_a - x_b, (p - q) mod L) f(b, q),
 *      with Neumaier-compensated accumulation;
 *   6. the plain DFT of the tabulated kernel along the line,
 *         g^k(d) = sum_s G~(d, s) exp(-2 pi i k s / L),
 *      used only to check the per-mode tables of the CUDA path.
 *
 * Build: any C11 compiler, with floating-point contraction disabled so that
 * the error-free transformations of the double-double helpers stay exact:
 *     cc -O2 -ffp-contract=off -fPIC -shared -pthread fbc_oracle.c -lm
 */

#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

typedef struct {
    int32_t kind;   /* 0: isotropic (Kelvin), 1: cubic (Barnett quadrature) */
    double mu, nu;  /* isotropic shear modulus and Poisson ratio */
    double C11, C12, C44; /* cubic constants in the crystal frame */
    double Q[9];    /* row-major rotation, r_crystal = Q r_computational */
    int32_t nquad;  /* Barnett trapezoid nodes on [0, pi) */
} orc_material;

/* ------------------------------------------------------------------ */
/* double-double helpers (Dekker / Knuth error-free transformations)   */
/* ------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;

static dd dd_from(double a) { dd r = {a, 0.0}; return r; }

static dd two_sum(double a, double b) {
    dd r;
    double s = a + b;
    double bb = s - a;
    r.hi = s;
    r.lo = (a - (s - bb)) + (b - bb);
    return r;
}

static dd fast_two_sum(double a, double b) {
    dd r;
    double s = a + b;
    r.hi = s;
    r.lo = b - (s - a);
    return r;
}

static dd dd_add_d(dd x, double b) {
    dd s = two_sum(x.hi, b);
    s.lo += x.lo;
    return fast_two_sum(s.hi, s.lo);
}

static dd dd_add(dd x, dd y) {
    dd s = two_sum(x.hi, y.hi);
    dd t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

static dd dd_mul_d(dd x, double b) {
    double p = x.hi * b;
    double e = fma(x.hi, b, -p);
    e += x.lo * b;
    return fast_two_sum(p, e);
}

static dd dd_div_d(dd x, double b) {
    double q1 = x.hi / b;
    dd r = dd_add(x, dd_mul_d(dd_from(q1), -b));
    double q2 = r.hi / b;
    return fast_two_sum(q1, q2);
}

/* ------------------------------------------------------------------ */
/* Step 1: continuum Green function of the infinite medium             */
/* ------------------------------------------------------------------ */

/* Kelvin's solution for a unit point force in an isotropic medium:
 *   G_ij(r) = [ (3 - 4 nu) delta_ij + r_i r_j / |r|^2 ] / (16 pi mu (1 - nu) |r|). */
static void green_kelvin(double mu, double nu, const double r[3], double G[9]) {
    double R2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double R = sqrt(R2);
    double pre = 1.0 / (16.0 * M_PI * mu * (1.0 - nu) * R);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            G[3 * i + j] = pre * ((i == j ? (3.0 - 4.0 * nu) : 0.0) + r[i] * r[j] / R2);
}

/* Full stiffness tensor C_ijkl (81 entries) of a cubic crystal, rotated into
 * the computational frame: C'_ijkl = Q_ai Q_bj Q_ck Q_dl C_abcd. */
static void cubic_stiffness(const orc_material* m, double Cr[81]) {
    double C[81];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) {
                    double v = 0.0;
                    if (i == j && k == l) v += m->C12;
                    if (i == k && j == l) v += m->C44;
                    if (i == l && j == k) v += m->C44;
                    if (i == j && j == k && k == l) v += m->C11 - m->C12 - 2.0 * m->C44;
                    C[27 * i + 9 * j + 3 * k + l] = v;
                }
    const double* Q = m->Q;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) {
                    double v = 0.0;
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            for (int c = 0; c < 3; c++)
                                for (int d = 0; d < 3; d++)
                                    v += Q[3 * a + i] * Q[3 * b + j] * Q[3 * c + k] * Q[3 * d + l] *
                                         C[27 * a + 9 * b + 3 * c + d];
                    Cr[27 * i + 9 * j + 3 * k + l] = v;
                }
}

/* Inverse of a general 3x3 matrix by the adjugate. */
static void inv3(const double A[9], double B[9]) {
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    double id = 1.0 / det;
    B[0] = c00 * id;
    B[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    B[3] = c01 * id;
    B[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    B[6] = c02 * id;
    B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
}

/* Barnett's representation of the anisotropic Green function:
 *   G(r) = 1 / (8 pi^2 |r|) * integral_0^{2 pi} (zz)^{-1} dpsi,
 *   (zz)_ik = C_ijkl z_j z_l,  z = cos(psi) e1 + sin(psi) e2,  {e1, e2} _|_ r.
 * The integrand has period pi, so the integral is 2 * integral_0^pi, taken
 * with the trapezoid rule on nquad equally spaced nodes. */
static void green_barnett(const double Cr[81], int nquad, const double r[3], double G[9]) {
    double R = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double rh[3] = {r[0] / R, r[1] / R, r[2] / R};
    /* e1: the coordinate axis least aligned with r_hat, made orthogonal */
    int ax = 0;
    if (fabs(rh[1]) < fabs(rh[ax])) ax = 1;
    if (fabs(rh[2]) < fabs(rh[ax])) ax = 2;
    double e1[3] = {0, 0, 0};
    e1[ax] = 1.0;
    double dot = rh[ax];
    for (int i = 0; i < 3; i++) e1[i] -= dot * rh[i];
    double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; i++) e1[i] /= n1;
    double e2[3] = {rh[1] * e1[2] - rh[2] * e1[1], rh[2] * e1[0] - rh[0] * e1[2],
                    rh[0] * e1[1] - rh[1] * e1[0]};
    double S[9] = {0};
    for (int q = 0; q < nquad; q++) {
        double psi = M_PI * (double)q / (double)nquad;
        double cp = cos(psi), sp = sin(psi);
        double z[3] = {cp * e1[0] + sp * e2[0], cp * e1[1] + sp * e2[1], cp * e1[2] + sp * e2[2]};
        double zz[9];
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++) zz[3 * j + l] = z[j] * z[l];
        double M[9], Mi[9];
        for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) {
                double v = 0.0;
                for (int j = 0; j < 3; j++)
                    for (int l = 0; l < 3; l++) v += Cr[27 * i + 9 * j + 3 * k + l] * zz[3 * j + l];
                M[3 * i + k] = v;
            }
        inv3(M, Mi);
        for (int t = 0; t < 9; t++) S[t] += Mi[t];
    }
    /* 2 * (pi / nquad) * S / (8 pi^2 R) */
    double pre = 2.0 * (M_PI / (double)nquad) / (8.0 * M_PI * M_PI * R);
    for (int t = 0; t < 9; t++) G[t] = pre * S[t];
}

typedef struct {
    int kind;
    double mu, nu;
    double Cr[81];
    int nquad;
} green_ctx;

static int green_ctx_init(const orc_material* m, green_ctx* g) {
    memset(g, 0, sizeof(*g));
    g->kind = m->kind;
    if (m->kind == 0) {
        if (!(m->mu > 0.0) || !(m->nu < 0.5) || !(m->nu > -1.0)) return ORC_EINVAL;
        g->mu = m->mu;
        g->nu = m->nu;
        return ORC_OK;
    }
    if (m->kind == 1) {
        if (m->nquad < 4) return ORC_EINVAL;
        cubic_stiffness(m, g->Cr);
        g->nquad = m->nquad;
        return ORC_OK;
    }
    return ORC_EINVAL;
}

static void green_eval(const green_ctx* g, const double r[3], double G[9]) {
    if (g->kind == 0)
        green_kelvin(g->mu, g->nu, r, G);
    else
        green_barnett(g->Cr, g->nquad, r, G);
}

int orc_green(const orc_material* m, const double r[3], double G[9]) {
    green_ctx g;
    int st = green_ctx_init(m, &g);
    if (st) return st;
    if (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0) return ORC_EINVAL;
    green_eval(&g, r, G);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Steps 2-3: regularised image sum and Richardson extrapolation      */
/* ------------------------------------------------------------------ */

/* Richardson weights w_i = (n+i)^N (-1)^{i+N} / (i! (N-i)!), i = 0..N. */
int orc_richardson_weights(int n, int N, double* w) {
    if (n < 1 || N < 0 || N > 16) return ORC_EINVAL;
    for (int i = 0; i <= N; i++) {
        double num = pow((double)(n + i), (double)N);
        double den = 1.0;
        for (int t = 2; t <= i; t++) den *= (double)t;
        for (int t = 2; t <= N - i; t++) den *= (double)t;
        double sgn = ((i + N) % 2) ? -1.0 : 1.0;
        w[i] = sgn * num / den;
    }
    return ORC_OK;
}

/* G(0, 0, m l3) + G(0, 0, -m l3) for m = 1..n+N: the terms Eq. 32 subtracts,
 * which do not depend on the evaluation point. */
static void reference_terms(const green_ctx* g, double l3, int m_last, double* ref /* [m_last][9] */) {
    double Gp[9], Gm[9];
    for (int m = 1; m <= m_last; m++) {
        double zp[3] = {0.0, 0.0, (double)m * l3};
        double zm[3] = {0.0, 0.0, -(double)m * l3};
        green_eval(g, zp, Gp);
        green_eval(g, zm, Gm);
        for (int t = 0; t < 9; t++) ref[(m - 1) * 9 + t] = Gp[t] + Gm[t];
    }
}

/* Q0 of Eq. 36 at point r for period l3, from the partial sums of Eq. 35.
 * Partial sums and the extrapolation are carried in double-double.  `ref`
 * holds the subtracted terms from reference_terms(). */
static void periodic_q0(const green_ctx* g, double l3, int n, int N, const double* ref, const double r[3],
                        double out[9]) {
    dd part[9];
    dd acc[9];
    double G[9];
    for (int t = 0; t < 9; t++) { acc[t] = dd_from(0.0); }
    /* i = 0 term: G(r), nothing subtracted */
    green_eval(g, r, G);
    for (int t = 0; t < 9; t++) part[t] = dd_from(G[t]);
    int m_last = n + N;
    for (int m = 1; m <= m_last; m++) {
        double rp[3] = {r[0], r[1], r[2] + (double)m * l3};
        double rm[3] = {r[0], r[1], r[2] - (double)m * l3};
        green_eval(g, rp, G);
        for (int t = 0; t < 9; t++) part[t] = dd_add_d(part[t], G[t]);
        green_eval(g, rm, G);
        for (int t = 0; t < 9; t++) part[t] = dd_add_d(part[t], G[t]);
        for (int t = 0; t < 9; t++) part[t] = dd_add_d(part[t], -ref[(m - 1) * 9 + t]);
        if (m >= n) {
            /* part now holds G_m; add its Richardson term (i = m - n) */
            int i = m - n;
            double num = pow((double)m, (double)N);
            double den = 1.0;
            for (int t = 2; t <= i; t++) den *= (double)t;
            for (int t = 2; t <= N - i; t++) den *= (double)t;
            double sgn = ((i + N) % 2) ? -1.0 : 1.0;
            for (int t = 0; t < 9; t++) {
                dd term = dd_div_d(dd_mul_d(part[t], sgn * num), den);
                acc[t] = dd_add(acc[t], term);
            }
        }
    }
    for (int t = 0; t < 9; t++) out[t] = acc[t].hi + acc[t].lo;
}

int orc_periodic(const orc_material* m, double l3, int n, int N, const double r[3], double out[9]) {
    green_ctx g;
    int st = green_ctx_init(m, &g);
    if (st) return st;
    if (!(l3 > 0.0) || n < 1 || N < 0 || N > 16 || n + N > 32) return ORC_EINVAL;
    if (r[0] == 0.0 && r[1] == 0.0) return ORC_EINVAL; /* on-axis: singular image */
    double ref[32 * 9];
    reference_terms(&g, l3, n + N, ref);
    periodic_q0(&g, l3, n, N, ref, r, out);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Thread pool helper: static work split by an atomic counter          */
/* ------------------------------------------------------------------ */
typedef void (*task_fn)(void* ctx, long item);
typedef struct {
    task_fn fn;
    void* ctx;
    long n_items;
    long next;
    pthread_mutex_t mu;
} pool_t;

static void* pool_worker(void* arg) {
    pool_t* p = (pool_t*)arg;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        long it = p->next++;
        pthread_mutex_unlock(&p->mu);
        if (it >= p->n_items) break;
        p->fn(p->ctx, it);
    }
    return NULL;
}

static void run_parallel(task_fn fn, void* ctx, long n_items, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pool_t p;
    p.fn = fn;
    p.ctx = ctx;
    p.n_items = n_items;
    p.next = 0;
    pthread_mutex_init(&p.mu, NULL);
    if (nthreads == 1) {
        pool_worker(&p);
    } else {
        pthread_t th[256];
        int started = 0;
        for (int t = 0; t < nthreads; t++)
            if (pthread_create(&th[t], NULL, pool_worker, &p) == 0) started++;
            else break;
        if (started == 0) pool_worker(&p);
        for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    }
    pthread_mutex_destroy(&p.mu);
}

/* ------------------------------------------------------------------ */
/* Step 4: tabulated periodic kernel G~(d, s), s = 0..L-1               */
/* ------------------------------------------------------------------ */
typedef struct {
    green_ctx g;
    int L;
    double c;
    int n, N;
    const int32_t* d;
    const double* ref; /* [n+N][9] */
    double* out; /* [nd][L][9] */
} table_ctx;

static void table_task(void* vctx, long item) {
    table_ctx* t = (table_ctx*)vctx;
    int L = t->L;
    long di = item / L;
    int s = (int)(item % L);
    double l3 = (double)L * t->c;
    double r[3] = {(double)t->d[2 * di], (double)t->d[2 * di + 1], 0.0};
    double* o = t->out + ((size_t)di * L + s) * 9;
    if (2 * s == L) {
        double a[9], b[9];
        r[2] = 0.5 * l3;
        periodic_q0(&t->g, l3, t->n, t->N, t->ref, r, a);
        r[2] = -0.5 * l3;
        periodic_q0(&t->g, l3, t->n, t->N, t->ref, r, b);
        for (int k = 0; k < 9; k++) o[k] = 0.5 * (a[k] + b[k]);
    } else {
        int sc = (2 * s < L) ? s : s - L;
        r[2] = (double)sc * t->c;
        periodic_q0(&t->g, l3, t->n, t->N, t->ref, r, o);
    }
}

int orc_kernel_table(const orc_material* m, int L, double c, int n, int N, int nd, const int32_t* d,
                     double* out, int nthreads) {
    table_ctx t;
    int st = green_ctx_init(m, &t.g);
    if (st) return st;
    if (L < 2 || (L % 2) || !(c > 0.0) || n < 1 || N < 0 || N > 16 || n + N > 32 || nd < 0) return ORC_EINVAL;
    for (int i = 0; i < nd; i++)
        if (d[2 * i] == 0 && d[2 * i + 1] == 0) return ORC_EINVAL;
    t.L = L;
    t.c = c;
    t.n = n;
    t.N = N;
    t.d = d;
    t.out = out;
    double ref[32 * 9];
    reference_terms(&t.g, (double)L * c, n + N, ref);
    t.ref = ref;
    run_parallel(table_task, &t, (long)nd * L, nthreads);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Step 5: real-space pad update at sampled pad atoms                   */
/* ------------------------------------------------------------------ */
typedef struct {
    int n_i, L;
    const int32_t* d_index; /* [n_samp_cols][n_i] index of x_a - x_b in the table */
    const double* table;    /* [nd][L][9] */
    int n_rhs;
    const double* f;        /* [n_rhs][n_i][L][3], already projected */
    const int32_t* samp_col;/* [n_samp] which row of d_index */
    const int32_t* samp_p;  /* [n_samp] repeat index p */
    int n_samp;
    double* u;              /* [n_rhs][n_samp][3] */
} apply_ctx;

static void apply_task(void* vctx, long item) {
    apply_ctx* A = (apply_ctx*)vctx;
    int rhs = (int)(item / A->n_samp);
    int smp = (int)(item % A->n_samp);
    int L = A->L;
    int p = A->samp_p[smp];
    const int32_t* didx = A->d_index + (size_t)A->samp_col[smp] * A->n_i;
    const double* f = A->f + (size_t)rhs * A->n_i * L * 3;
    /* Neumaier summation per component */
    double sum[3] = {0, 0, 0}, comp[3] = {0, 0, 0};
    for (int b = 0; b < A->n_i; b++) {
        const double* Gd = A->table + (size_t)didx[b] * L * 9;
        const double* fb = f + (size_t)b * L * 3;
        for (int q = 0; q < L; q++) {
            int s = p - q;
            if (s < 0) s += L;
            const double* G = Gd + (size_t)s * 9;
            const double* fq = fb + (size_t)q * 3;
            for (int i = 0; i < 3; i++) {
                for (int j = 0; j < 3; j++) {
                    double x = G[3 * i + j] * fq[j];
                    double tsum = sum[i] + x;
                    if (fabs(sum[i]) >= fabs(x))
                        comp[i] += (sum[i] - tsum) + x;
                    else
                        comp[i] += (x - tsum) + sum[i];
                    sum[i] = tsum;
                }
            }
        }
    }
    double* uo = A->u + ((size_t)rhs * A->n_samp + smp) * 3;
    for (int i = 0; i < 3; i++) uo[i] = sum[i] + comp[i];
}

int orc_apply_samples(int n_i, int L, int n_cols, const int32_t* d_index, int nd, const double* table,
                      int n_rhs, const double* f, int n_samp, const int32_t* samp_col, const int32_t* samp_p,
                      double* u, int nthreads) {
    if (n_i < 0 || L < 1 || n_cols < 0 || nd < 0 || n_rhs < 0 || n_samp < 0) return ORC_EINVAL;
    for (long t = 0; t < (long)n_cols * n_i; t++)
        if (d_index[t] < 0 || d_index[t] >= nd) return ORC_EINVAL;
    for (int s = 0; s < n_samp; s++)
        if (samp_col[s] < 0 || samp_col[s] >= n_cols || samp_p[s] < 0 || samp_p[s] >= L) return ORC_EINVAL;
    apply_ctx A = {n_i, L, d_index, table, n_rhs, f, samp_col, samp_p, n_samp, u};
    run_parallel(apply_task, &A, (long)n_rhs * n_samp, nthreads);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Step 6: plain DFT of the tabulated kernel along the line             */
/* ------------------------------------------------------------------ */
typedef struct {
    int L, K;
    const double* table; /* [nd][L][9] */
    double* re;          /* [nd][K][9] */
    double* im;
} dft_ctx;

static void dft_task(void* vctx, long item) {
    dft_ctx* D = (dft_ctx*)vctx;
    int L = D->L, K = D->K;
    long di = item / K;
    int k = (int)(item % K);
    const double* T = D->table + (size_t)di * L * 9;
    dd sr[9], si[9];
    for (int t = 0; t < 9; t++) { sr[t] = dd_from(0.0); si[t] = dd_from(0.0); }
    for (int s = 0; s < L; s++) {
        long ks = ((long)k * s) % L;
        double ang = 2.0 * M_PI * (double)ks / (double)L;
        double cs = cos(ang), sn = sin(ang);
        for (int t = 0; t < 9; t++) {
            sr[t] = dd_add(sr[t], dd_mul_d(dd_from(T[s * 9 + t]), cs));
            si[t] = dd_add(si[t], dd_mul_d(dd_from(T[s * 9 + t]), -sn));
        }
    }
    for (int t = 0; t < 9; t++) {
        D->re[((size_t)di * K + k) * 9 + t] = sr[t].hi + sr[t].lo;
        D->im[((size_t)di * K + k) * 9 + t] = si[t].hi + si[t].lo;
    }
}

int orc_mode_table(int L, int nd, const double* table, double* re, double* im, int nthreads) {
    if (L < 2 || (L % 2) || nd < 0) return ORC_EINVAL;
    dft_ctx D = {L, L / 2 + 1, table, re, im};
    run_parallel(dft_task, &D, (long)nd * D.K, nthreads);
    return ORC_OK;
}
