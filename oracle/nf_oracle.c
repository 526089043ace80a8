/*
 * Plain FP64 CPU oracle for the Abacus near-field force
 * (Garrison et al., "The Abacus Cosmological N-body Code").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference
 * that the CUDA path is checked against.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no source, header,
 * table or helper with the CUDA library, and it must be compiled without FMA
 * contraction (-ffp-contract=off) so that every FP64 operation in the binning
 * is a single correctly rounded IEEE operation.
 *
 * What it computes, and where the paper defines it:
 *   - Binning into a periodic K^3 grid of cells, with positions stored as
 *     FP32 offsets from the cell centre (Sec. "Force Accuracy", overview:
 *     cell-centred single-precision offsets; Sec. "Two-Stage Execution": the
 *     K^3 grid).  Cells are numbered (cx*K + cy)*K + cz; particles in a cell
 *     keep their input order (a stable counting sort).
 *   - The near-field acceleration: every particle receives the direct force
 *     from every particle in the (2R+1)^3 cells around its own cell, with open
 *     boundaries, the source image taken in the unwrapped neighbour cell
 *     (Sec. "Force Solver": exact near/far split; Sec. "GPU Near-Field
 *     Computation": the 5^3 neighbour cells).
 *   - The spline-softened pair force of Eq. (spline), Sec. "Force Softening":
 *       F(r) = [10 - 15 u + 6 u^2] r_vec / eps_s^3   for u = r/eps_s < 1,
 *       F(r) = r_vec / r^3                           otherwise,
 *     with eps_s = 2.16 eps_p (same section), eps_p the Plummer-equivalent
 *     softening the caller passes.  G = 1 and every particle has mass 1/N.
 *     The force is attractive: the acceleration of i points towards j.
 *   - The apodized top-hat density estimate the paper's kernel accumulates as
 *     a 4th component (Sec. "Force Kernel"): rho_i = sum over near-field j
 *     with r_ij < b of (1 - r_ij^2 / b^2), the particle itself included
 *     (it contributes 1).  The kernel accumulates b^2 - r^2; this is that sum
 *     divided by b^2.
 *   - Cell multipoles in the complete basis, Eq. (multipoles) in Sec.
 *     "Computation of the Cell Multipoles": M^{abc} = sum_q x_q^a y_q^b z_q^c
 *     over the particles of a cell, a + b + c <= p, with (x, y, z) the
 *     displacement from the cell centre in box units (unit masses), taken
 *     from the particle's stored FP32 cell-centred offset times the cell
 *     width: the paper's particle state is that offset (Sec. "Force
 *     Accuracy", overview).
 *   - The adjoint (the gradient of L = sum_i g_i . a_i with respect to the
 *     positions), which the paper does not give; it is the derivative of the
 *     sum above: dL/dx_i = m sum_j J(d_ij) (g_j - g_i) with J(d) the Jacobian
 *     of F, J = f I + (f'/r) d d^T.
 *
 * The two branches of Eq. (spline) are evaluated with a plain branch here, not
 * with the min() form the paper's kernel uses (Sec. "Force Kernel").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_EPS_RATIO 2.16 /* eps_s / eps_p, Sec. "Force Softening" */

/* ------------------------------------------------------------------------- */
/* Binning                                                                    */
/* ------------------------------------------------------------------------- */

/* One coordinate: t = x * (K / box) in FP64, c = floor(t), offset from the
 * centre of cell c in cell units is (t - c) - 0.5, rounded once to FP32; the
 * cell index wraps periodically, c mod K in [0, K).  `wrap` returns the number
 * of whole boxes between the input coordinate and its image in [0, box). */
int oracle_coord(float x, double kl, int K, int *cell, float *offset,
                        double *wrap)
{
    double xd = (double)x;
    if (!isfinite(xd)) return 1;
    double t = xd * kl;
    double c = floor(t);
    double frac = t - c;
    double off = frac - 0.5;
    double cm = fmod(c, (double)K);
    if (cm < 0.0) cm += (double)K;
    *cell = (int)cm;
    *offset = (float)off;
    *wrap = (c - cm) / (double)K;
    return 0;
}

/* Bins N positions.  Outputs (all caller-allocated):
 *   cell_offsets[K^3 + 1]: first sorted slot of every cell, last entry = N;
 *   rel[4*N]: sorted (offset_x, offset_y, offset_z, bits of original index);
 *   perm[N]: sorted slot -> original index;
 *   cell_of[N] (may be NULL): cell of every particle, in input order.
 * Returns the number of non-finite positions (0 on success). */
int64_t oracle_bin(const float *pos, int64_t N, double box, int K,
                   int32_t *cell_offsets, float *rel, int32_t *perm,
                   int32_t *cell_of)
{
    const double kl = (double)K / box;
    const int64_t ncell = (int64_t)K * K * K;
    int32_t *cid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    float *off = (float *)malloc(sizeof(float) * 3 * (size_t)(N > 0 ? N : 1));
    int64_t *count = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t bad = 0;
    for (int64_t i = 0; i < N; ++i) {
        int c[3];
        double w;
        for (int d = 0; d < 3; ++d) {
            if (oracle_coord(pos[3 * i + d], kl, K, &c[d], &off[3 * i + d], &w)) {
                bad++;
                c[d] = 0;
                off[3 * i + d] = 0.0f;
            }
        }
        cid[i] = (int32_t)(((int64_t)c[0] * K + c[1]) * K + c[2]);
        count[cid[i]]++;
    }
    /* exclusive prefix sum -> first slot of each cell */
    int64_t run = 0;
    for (int64_t c = 0; c < ncell; ++c) {
        int64_t n = count[c];
        cell_offsets[c] = (int32_t)run;
        count[c] = run;
        run += n;
    }
    cell_offsets[ncell] = (int32_t)run;
    /* stable scatter in input order */
    for (int64_t i = 0; i < N; ++i) {
        int64_t s = count[cid[i]]++;
        perm[s] = (int32_t)i;
        rel[4 * s + 0] = off[3 * i + 0];
        rel[4 * s + 1] = off[3 * i + 1];
        rel[4 * s + 2] = off[3 * i + 2];
        int32_t bits = (int32_t)i;
        memcpy(&rel[4 * s + 3], &bits, sizeof(bits));
        if (cell_of) cell_of[i] = cid[i];
    }
    free(cid);
    free(off);
    free(count);
    return bad;
}

/* ------------------------------------------------------------------------- */
/* Shared set-up for the force sums                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t N;
    int K, R;
    double box, eps_s, m;
    int32_t *offsets; /* [K^3+1] */
    int32_t *order;   /* sorted slot -> original index */
    int32_t *cell;    /* [N][3] cell coordinates */
    double *xw;       /* [N][3] positions moved into [0, box) by whole boxes */
} oracle_grid;

static int oracle_grid_init(oracle_grid *g, const float *pos, int64_t N, double box,
                            int K, int R, double eps_p)
{
    memset(g, 0, sizeof(*g));
    g->N = N;
    g->K = K;
    g->R = R;
    g->box = box;
    g->eps_s = ORACLE_EPS_RATIO * eps_p;
    g->m = 1.0 / (double)N;
    const int64_t ncell = (int64_t)K * K * K;
    g->offsets = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
    g->order = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    g->cell = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)N);
    g->xw = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    float *rel = (float *)malloc(sizeof(float) * 4 * (size_t)N);
    int64_t bad = oracle_bin(pos, N, box, K, g->offsets, rel, g->order, NULL);
    free(rel);
    if (bad) return 1;
    const double kl = (double)K / box;
    for (int64_t i = 0; i < N; ++i) {
        for (int d = 0; d < 3; ++d) {
            int c = 0;
            float o = 0.0f;
            double w = 0.0;
            oracle_coord(pos[3 * i + d], kl, K, &c, &o, &w);
            g->cell[3 * i + d] = c;
            g->xw[3 * i + d] = (double)pos[3 * i + d] - w * box;
        }
    }
    return 0;
}

static void oracle_grid_free(oracle_grid *g)
{
    free(g->offsets);
    free(g->order);
    free(g->cell);
    free(g->xw);
}

/* f(r) of Eq. (spline), written so that F(d) = f(|d|) d. */
static double spline_f(double r, double eps_s)
{
    if (r < eps_s) {
        double u = r / eps_s;
        return (10.0 - 15.0 * u + 6.0 * u * u) / (eps_s * eps_s * eps_s);
    }
    return 1.0 / (r * r * r);
}

/* f'(r)/r, the radial part of the Jacobian of F.  Eq. (spline) gives
 * f' = (-15 + 12 u) / eps_s^4 inside the softening and -3/r^4 outside. */
static double spline_fprime_over_r(double r, double eps_s)
{
    if (r < eps_s) {
        double u = r / eps_s;
        double e4 = eps_s * eps_s * eps_s * eps_s;
        return (12.0 * u - 15.0) / (e4 * eps_s * u);
    }
    double r2 = r * r;
    return -3.0 / (r2 * r2 * r);
}

/* Visits every source j in the (2R+1)^3 neighbour cells of particle i, with the
 * separation d = x_j(image) - x_i in FP64 (position of i taken from `xi`). */
typedef void (*pair_visitor)(void *ctx, int64_t j, const double d[3]);

static void visit_neighbours(const oracle_grid *g, const int32_t cell_i[3],
                             const double xi[3], pair_visitor fn, void *ctx)
{
    const int K = g->K, R = g->R;
    for (int a = -R; a <= R; ++a)
        for (int b = -R; b <= R; ++b)
            for (int c = -R; c <= R; ++c) {
                int u[3] = {cell_i[0] + a, cell_i[1] + b, cell_i[2] + c};
                int n[3];
                double shift[3];
                for (int k = 0; k < 3; ++k) {
                    n[k] = ((u[k] % K) + K) % K;
                    /* the source image sits in the unwrapped neighbour cell */
                    shift[k] = (double)((u[k] - n[k]) / K) * g->box;
                }
                int64_t cid = ((int64_t)n[0] * K + n[1]) * K + n[2];
                for (int32_t s = g->offsets[cid]; s < g->offsets[cid + 1]; ++s) {
                    int64_t j = g->order[s];
                    double d[3];
                    for (int k = 0; k < 3; ++k)
                        d[k] = (g->xw[3 * j + k] + shift[k]) - xi[k];
                    fn(ctx, j, d);
                }
            }
}

/* ------------------------------------------------------------------------- */
/* Forces                                                                     */
/* ------------------------------------------------------------------------- */

typedef struct {
    double eps_s;
    double a[3];
} force_ctx;

static void force_visit(void *vctx, int64_t j, const double d[3])
{
    (void)j;
    force_ctx *ctx = (force_ctx *)vctx;
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double f = spline_f(r, ctx->eps_s);
    ctx->a[0] += f * d[0];
    ctx->a[1] += f * d[1];
    ctx->a[2] += f * d[2];
}

static void force_on(const oracle_grid *g, int64_t i, double out[3])
{
    force_ctx ctx = {g->eps_s, {0.0, 0.0, 0.0}};
    visit_neighbours(g, &g->cell[3 * i], &g->xw[3 * i], force_visit, &ctx);
    out[0] = g->m * ctx.a[0];
    out[1] = g->m * ctx.a[1];
    out[2] = g->m * ctx.a[2];
}

/* Near-field accelerations of the listed sinks on a binned grid. */
static void grid_forces(const oracle_grid *g, const int64_t *sinks, int64_t n, double *out, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int64_t q = 0; q < n; ++q) {
        int64_t i = sinks ? sinks[q] : q;
        force_on(g, i, &out[3 * q]);
    }
}

/* Near-field accelerations of the `nsinks` particles listed in `sinks`
 * (or of all N particles when sinks == NULL), FP64 out[nsinks][3].
 * nthreads <= 0 uses every OpenMP thread.  Returns 0, or 1 on non-finite input. */
int oracle_forces(const float *pos, int64_t N, double box, int K, int R, double eps_p,
                  const int64_t *sinks, int64_t nsinks, double *out, int nthreads)
{
    oracle_grid g;
    if (oracle_grid_init(&g, pos, N, box, K, R, eps_p)) {
        oracle_grid_free(&g);
        return 1;
    }
    grid_forces(&g, sinks, sinks ? nsinks : N, out, nthreads);
    oracle_grid_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint                                                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    double eps_s;
    const double *g;
    double gi[3];
    double out[3];
} adj_ctx;

static void adj_visit(void *vctx, int64_t j, const double d[3])
{
    adj_ctx *ctx = (adj_ctx *)vctx;
    double v[3] = {ctx->g[3 * j + 0] - ctx->gi[0], ctx->g[3 * j + 1] - ctx->gi[1],
                   ctx->g[3 * j + 2] - ctx->gi[2]};
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double f = spline_f(r, ctx->eps_s);
    double fr = 0.0; /* J(0) = f(0) I: the d d^T term vanishes */
    if (r > 0.0) fr = spline_fprime_over_r(r, ctx->eps_s);
    double dv = d[0] * v[0] + d[1] * v[1] + d[2] * v[2];
    for (int k = 0; k < 3; ++k) ctx->out[k] += f * v[k] + fr * dv * d[k];
}

/* dL/dx at the listed sinks on a binned grid. */
static void grid_adjoint(const oracle_grid *g, const double *gvec, const int64_t *sinks, int64_t n, double *out,
                         int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int64_t q = 0; q < n; ++q) {
        int64_t i = sinks ? sinks[q] : q;
        adj_ctx ctx;
        ctx.eps_s = g->eps_s;
        ctx.g = gvec;
        for (int k = 0; k < 3; ++k) {
            ctx.gi[k] = gvec[3 * i + k];
            ctx.out[k] = 0.0;
        }
        visit_neighbours(g, &g->cell[3 * i], &g->xw[3 * i], adj_visit, &ctx);
        for (int k = 0; k < 3; ++k) out[3 * q + k] = g->m * ctx.out[k];
    }
}

/* dL/dx for L = sum_i g_i . a_i, at the listed particles (or all).  g is FP64
 * [N][3] in input order; out is FP64 [nsinks][3]. */
int oracle_adjoint(const float *pos, const double *gvec, int64_t N, double box, int K,
                   int R, double eps_p, const int64_t *sinks, int64_t nsinks,
                   double *out, int nthreads)
{
    oracle_grid g;
    if (oracle_grid_init(&g, pos, N, box, K, R, eps_p)) {
        oracle_grid_free(&g);
        return 1;
    }
    grid_adjoint(&g, gvec, sinks, sinks ? nsinks : N, out, nthreads);
    oracle_grid_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* A binned grid kept between calls                                           */
/* ------------------------------------------------------------------------- */

/* The same set-up as oracle_forces/oracle_adjoint (binning, cell coordinates,
 * wrapped positions), done once so that several sink samples of one particle
 * set can be evaluated without binning it again.  Returns NULL on non-finite
 * input or when memory runs out. */
void *oracle_grid_new(const float *pos, int64_t N, double box, int K, int R, double eps_p)
{
    oracle_grid *g = (oracle_grid *)malloc(sizeof(oracle_grid));
    if (!g) return NULL;
    if (oracle_grid_init(g, pos, N, box, K, R, eps_p) || !g->offsets || !g->order || !g->cell || !g->xw) {
        oracle_grid_free(g);
        free(g);
        return NULL;
    }
    return g;
}

void oracle_grid_delete(void *g)
{
    if (!g) return;
    oracle_grid_free((oracle_grid *)g);
    free(g);
}

/* Cell offsets [K^3 + 1] and sorted slot -> original index [N] of the grid. */
void oracle_grid_binning(const void *vg, int32_t *offsets, int32_t *order)
{
    const oracle_grid *g = (const oracle_grid *)vg;
    const int64_t ncell = (int64_t)g->K * g->K * g->K;
    memcpy(offsets, g->offsets, sizeof(int32_t) * (size_t)(ncell + 1));
    memcpy(order, g->order, sizeof(int32_t) * (size_t)g->N);
}

void oracle_grid_forces(const void *g, const int64_t *sinks, int64_t nsinks, double *out, int nthreads)
{
    grid_forces((const oracle_grid *)g, sinks, nsinks, out, nthreads);
}

void oracle_grid_adjoint(const void *g, const double *gvec, const int64_t *sinks, int64_t nsinks, double *out,
                         int nthreads)
{
    grid_adjoint((const oracle_grid *)g, gvec, sinks, nsinks, out, nthreads);
}

/* ------------------------------------------------------------------------- */
/* Top-hat density estimate                                                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    double b;
    double rho;
} dens_ctx;

static void dens_visit(void *vctx, int64_t j, const double d[3])
{
    (void)j;
    dens_ctx *ctx = (dens_ctx *)vctx;
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (r < ctx->b) ctx->rho += 1.0 - (r * r) / (ctx->b * ctx->b);
}

/* rho_i = sum_{j in N(i), r_ij < b} (1 - r_ij^2/b^2) at the listed particles
 * (or all), FP64 out[nsinks].  b in box units. */
int oracle_density(const float *pos, int64_t N, double box, int K, int R, double b,
                   const int64_t *sinks, int64_t nsinks, double *out, int nthreads)
{
    oracle_grid g;
    if (oracle_grid_init(&g, pos, N, box, K, R, 1.0)) {
        oracle_grid_free(&g);
        return 1;
    }
    int64_t n = sinks ? nsinks : N;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int64_t q = 0; q < n; ++q) {
        int64_t i = sinks ? sinks[q] : q;
        dens_ctx ctx = {b, 0.0};
        visit_neighbours(&g, &g.cell[3 * i], &g.xw[3 * i], dens_visit, &ctx);
        out[q] = ctx.rho;
    }
    oracle_grid_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Cell multipoles (complete basis)                                           */
/* ------------------------------------------------------------------------- */

/* Number of complete-basis terms of order p: (p+3)(p+2)(p+1)/6. */
int64_t oracle_multipole_terms(int p)
{
    return (int64_t)(p + 3) * (p + 2) * (p + 1) / 6;
}

/* M[cell][term] for every cell, terms ordered a (0..p), then b (0..p-a), then
 * c (0..p-a-b).  The displacement of a particle from its cell centre is its
 * FP32 cell-centred offset (the binning above) times box / K, in FP64. */
int oracle_multipoles(const float *pos, int64_t N, double box, int K, int p, double *M)
{
    const int64_t nt = oracle_multipole_terms(p);
    const int64_t ncell = (int64_t)K * K * K;
    memset(M, 0, sizeof(double) * (size_t)(ncell * nt));
    const double kl = (double)K / box;
    const double w = box / (double)K;
    for (int64_t i = 0; i < N; ++i) {
        int cell[3];
        double disp[3];
        for (int d = 0; d < 3; ++d) {
            int c = 0;
            float o = 0.0f;
            double wrap = 0.0;
            if (oracle_coord(pos[3 * i + d], kl, K, &c, &o, &wrap)) return 1;
            cell[d] = c;
            disp[d] = (double)o * w;
        }
        double *m = &M[(((int64_t)cell[0] * K + cell[1]) * K + cell[2]) * nt];
        int64_t t = 0;
        for (int a = 0; a <= p; ++a)
            for (int b = 0; b <= p - a; ++b)
                for (int c = 0; c <= p - a - b; ++c) {
                    double v = 1.0;
                    for (int e = 0; e < a; ++e) v *= disp[0];
                    for (int e = 0; e < b; ++e) v *= disp[1];
                    for (int e = 0; e < c; ++e) v *= disp[2];
                    m[t++] += v;
                }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Local energy for finite differences                                       */
/* ------------------------------------------------------------------------- */

typedef struct {
    double eps_s;
    const double *g;
    int64_t k;
    double gk[3];
    double sum;
} le_ctx;

static void le_visit(void *vctx, int64_t j, const double d[3])
{
    le_ctx *ctx = (le_ctx *)vctx;
    if (j == ctx->k) return; /* the self pair carries F(0) = 0 */
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double f = spline_f(r, ctx->eps_s);
    for (int q = 0; q < 3; ++q)
        ctx->sum += (ctx->gk[q] - ctx->g[3 * j + q]) * f * d[q];
}

/* The part of L = sum_i g_i . a_i that depends on particle k, with k moved to
 * the FP64 position xk (same periodic frame as its wrapped input position) and
 * every cell assignment frozen at the binning of the unmoved positions:
 *   L_k = m sum_{j in N(k)} (g_k - g_j) . F(x_j - x_k),
 * which uses F(-d) = -F(d) for the terms of a_j that involve k. */
int oracle_local_energy(const float *pos, const double *gvec, int64_t N, double box,
                        int K, int R, double eps_p, const int64_t *ks, int64_t nk,
                        const double *xk, double *out)
{
    oracle_grid g;
    if (oracle_grid_init(&g, pos, N, box, K, R, eps_p)) {
        oracle_grid_free(&g);
        return 1;
    }
    for (int64_t q = 0; q < nk; ++q) {
        le_ctx ctx;
        ctx.eps_s = g.eps_s;
        ctx.g = gvec;
        ctx.k = ks[q];
        ctx.sum = 0.0;
        for (int c = 0; c < 3; ++c) ctx.gk[c] = gvec[3 * ks[q] + c];
        visit_neighbours(&g, &g.cell[3 * ks[q]], &xk[3 * q], le_visit, &ctx);
        out[q] = g.m * ctx.sum;
    }
    oracle_grid_free(&g);
    return 0;
}

/* Wrapped FP64 positions used by the force sums (input minus whole boxes). */
int oracle_wrapped_positions(const float *pos, int64_t N, double box, int K, double *xw)
{
    const double kl = (double)K / box;
    for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) {
            int c = 0;
            float o = 0.0f;
            double w = 0.0;
            if (oracle_coord(pos[3 * i + d], kl, K, &c, &o, &w)) return 1;
            xw[3 * i + d] = (double)pos[3 * i + d] - w * box;
        }
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
