/*
 * Plain FP64 CPU oracle for the Abacus far field
 * (Garrison et al., "The Abacus Cosmological N-body Code", Sec. "Far-field
 * Computation").
 *
 * TEST INFRASTRUCTURE ONLY.  Like nf_oracle.c, this file is the slow,
 * obviously correct reference the CUDA path is checked against; only the
 * tests, the smoke check and the benchmark's CPU leg may load it, and it
 * shares nothing with the CUDA library.
 *
 * Notation.  Box side L, V = L^3, cell width w = L/K, unit masses (the
 * caller applies m = 1/N and G = 1).  Terms (a,b,c) of the complete basis
 * with a + b + c <= p are ordered a (0..p), then b (0..p-a), then
 * c (0..p-a-b), as the multipoles of Eq. (multipoles).
 *
 * What it computes:
 *   - The derivatives tensor.  For every cell offset g on the K^3 grid
 *     (sink cell minus source cell, mod K), D^{abc}(g) is the (a,b,c)-th
 *     Cartesian derivative, at the cell-centre separation, of the periodic
 *     potential of a unit mass: every periodic image, with the uniform
 *     neutralising background that Ewald summation implies, minus the one
 *     image the near field computes directly (an offset whose three
 *     components, taken in (-K/2, K/2], all lie in [-R, R]).  The paper: the
 *     derivatives include all periodic images, the near-field cells' images
 *     included, so the total force equals Ewald summation up to the finite
 *     multipole order (Sec. "Far-field Computation", overview).
 *     Ewald's split with parameter alpha (P. P. Ewald 1921):
 *         sum_n 1/|r + nL| -> sum_n erfc(alpha |r+nL|)/|r+nL|
 *                             + (4 pi/V) sum_{k != 0} exp(-k^2/4alpha^2)/k^2 cos(k.r)
 *                             - pi / (alpha^2 V),          k = 2 pi h / L.
 *     Cartesian derivatives of a radial function g(r) come from the Hermite
 *     recursion of McMurchie & Davidson (J. Comput. Phys. 26, 218, 1978):
 *     with g_m = (r^-1 d/dr)^m g and R^m_{tuv} the (t,u,v) derivative of g_m,
 *         R^m_{t+1,u,v} = t R^{m+1}_{t-1,u,v} + X R^{m+1}_{t,u,v}
 *     (likewise in Y and Z), and R^0_{abc} is the wanted derivative.  For
 *     erfc(alpha r)/r, g_m = (-1)^m B_m with B_0 = erfc(alpha r)/r and
 *         B_m = [(2m-1) B_{m-1} + (2 alpha^2)^m exp(-alpha^2 r^2)/(alpha sqrt(pi))] / r^2
 *     (W. Smith, CCP5 Newsletter 46, 1998).  The near image is removed as
 *     1/r = erfc(alpha r)/r + erf(alpha r)/r: its erfc part is left out of
 *     the image sum and its erf part, smooth at r = 0, is subtracted with
 *         g_m = (2/sqrt(pi)) (-2)^m sum_j (-r^2)^j alpha^(2m+2j+1) / (j! (2m+2j+1)),
 *     the series of (2/sqrt(pi)) int_0^alpha (-2t^2)^m exp(-t^2 r^2) dt.
 *   - The Taylors by the direct cyclic convolution over cells (the plain
 *     definition the FFT route must reproduce):
 *         T^n(c) = sum_{c'} sum_k (-1)^{|k|} / (n! k!) D^{n+k}(c - c') M^k(c'),
 *     |n| + |k| <= p, n! = n_x! n_y! n_z!.  This is the Taylor expansion of
 *     1/|Delta + x - s| in the sink displacement x and the source
 *     displacement s about the cell-centre separation Delta.
 *   - The far-field acceleration from the Taylors: the potential in a cell
 *     is -sum_n T^n x^n (unit masses, G = 1), so a = sum_n T^n grad(x^n),
 *     with x the particle's displacement from its cell centre (its stored
 *     FP32 cell-centred offset times w).
 *   - Reference forces by plain Ewald summation over every particle pair
 *     (the paper's Sec. "Force Accuracy" compares Abacus against Ewald
 *     sums): a_i = sum_{j != i} grad Phi(x_i - x_j) with Phi the Ewald sum
 *     above (no multipole expansion, no near/far split, no softening).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_coord(float x, double kl, int K, int *cell, float *offset, double *wrap);

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* position of term (a,b,c) in the complete-basis order of order p */
static int term_index(int a, int b, int c, int p)
{
    int t = 0;
    for (int a2 = 0; a2 < a; ++a2) t += (p - a2 + 1) * (p - a2 + 2) / 2;
    for (int b2 = 0; b2 < b; ++b2) t += p - a - b2 + 1;
    return t + c;
}

static int64_t nterms(int p) { return (int64_t)(p + 3) * (p + 2) * (p + 1) / 6; }

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* Hermite recursion: given g_m(r) for m = 0..p at r = (X, Y, Z), writes the
 * (a,b,c) derivative of g_0 for every term into out[nterms(p)] (added, times
 * `scale`).  cur/nxt are scratch arrays of (p+1)^3 doubles. */
static void hermite_add(int p, double X, double Y, double Z, const double *gm, double scale, double *out,
                        double *cur, double *nxt)
{
    const int P1 = p + 1;
#define IDX(t, u, v) (((t) * P1 + (u)) * P1 + (v))
    /* layer m = p: only R^p_{000} */
    nxt[IDX(0, 0, 0)] = gm[p];
    for (int m = p - 1; m >= 0; --m) {
        const int top = p - m;
        for (int t = 0; t <= top; ++t)
            for (int u = 0; u <= top - t; ++u)
                for (int v = 0; v <= top - t - u; ++v) {
                    double r;
                    if (t == 0 && u == 0 && v == 0)
                        r = gm[m];
                    else if (t > 0)
                        r = (t >= 2 ? (t - 1) * nxt[IDX(t - 2, u, v)] : 0.0) + X * nxt[IDX(t - 1, u, v)];
                    else if (u > 0)
                        r = (u >= 2 ? (u - 1) * nxt[IDX(t, u - 2, v)] : 0.0) + Y * nxt[IDX(t, u - 1, v)];
                    else
                        r = (v >= 2 ? (v - 1) * nxt[IDX(t, u, v - 2)] : 0.0) + Z * nxt[IDX(t, u, v - 1)];
                    cur[IDX(t, u, v)] = r;
                }
        double *sw = cur;
        cur = nxt;
        nxt = sw;
    }
    /* after the last swap the m = 0 layer is in nxt */
    int64_t q = 0;
    for (int a = 0; a <= p; ++a)
        for (int b = 0; b <= p - a; ++b)
            for (int c = 0; c <= p - a - b; ++c) out[q++] += scale * nxt[IDX(a, b, c)];
#undef IDX
}

/* g_m of erfc(alpha r)/r, m = 0..p, at r > 0 */
static void gm_erfc(int p, double alpha, double r, double *gm)
{
    const double r2 = r * r;
    const double e = exp(-alpha * alpha * r2) / (alpha * sqrt(M_PI));
    double B = erfc(alpha * r) / r;
    double pw = 1.0; /* (2 alpha^2)^m */
    gm[0] = B;
    for (int m = 1; m <= p; ++m) {
        pw *= 2.0 * alpha * alpha;
        B = ((2 * m - 1) * B + pw * e) / r2;
        gm[m] = (m & 1) ? -B : B;
    }
}

/* g_m of erf(alpha r)/r, m = 0..p, at any r >= 0 (the power series) */
static void gm_erf(int p, double alpha, double r, double *gm)
{
    const double x = -r * r;
    for (int m = 0; m <= p; ++m) {
        double sum = 0.0, term = 1.0; /* term = x^j / j! */
        double ap = pow(alpha, 2 * m + 1);
        for (int j = 0; j < 200; ++j) {
            const double add = term * ap / (double)(2 * m + 2 * j + 1);
            sum += add;
            if (j > 4 && fabs(add) < 1e-18 * fabs(sum)) break;
            term *= x / (double)(j + 1);
            ap *= alpha * alpha;
        }
        gm[m] = (2.0 / sqrt(M_PI)) * pow(-2.0, m) * sum;
    }
}

/* g_m of 1/r: (-1)^m (2m-1)!! / r^(2m+1) */
static void gm_coulomb(int p, double r, double *gm)
{
    double v = 1.0 / r;
    const double ir2 = 1.0 / (r * r);
    gm[0] = v;
    for (int m = 1; m <= p; ++m) {
        v *= -(double)(2 * m - 1) * ir2;
        gm[m] = v;
    }
}

static int centred(int g, int K) { return 2 * g > K ? g - K : g; }

/* D[g][term] for every cell offset g = (gx*K + gy)*K + gz.  alpha in 1/length;
 * real-space images n in [-nimg, nimg]^3, reciprocal vectors h in
 * [-hmax, hmax]^3 \ {0}. */
int oracle_derivatives(int K, int R, int p, double box, double alpha, int nimg, int hmax, double *D)
{
    const int64_t nt = nterms(p);
    const double w = box / (double)K;
    const double V = box * box * box;
    const int64_t ncell = (int64_t)K * K * K;
    const int H = 2 * hmax + 1;
    const int64_t nh = (int64_t)H * H * H;
    /* per reciprocal vector: weight and powers of k */
    double *kw = (double *)malloc(sizeof(double) * (size_t)nh);
    double *kv = (double *)malloc(sizeof(double) * 3 * (size_t)nh);
    for (int64_t q = 0; q < nh; ++q) {
        const int hx = (int)(q / (H * H)) - hmax, hy = (int)((q / H) % H) - hmax, hz = (int)(q % H) - hmax;
        const double kx = 2.0 * M_PI * hx / box, ky = 2.0 * M_PI * hy / box, kz = 2.0 * M_PI * hz / box;
        const double k2 = kx * kx + ky * ky + kz * kz;
        kv[3 * q] = kx;
        kv[3 * q + 1] = ky;
        kv[3 * q + 2] = kz;
        kw[q] = (hx == 0 && hy == 0 && hz == 0) ? 0.0 : (4.0 * M_PI / V) * exp(-k2 / (4.0 * alpha * alpha)) / k2;
    }
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        const int P1 = p + 1;
        double *cur = (double *)malloc(sizeof(double) * (size_t)P1 * P1 * P1);
        double *nxt = (double *)malloc(sizeof(double) * (size_t)P1 * P1 * P1);
        double *gm = (double *)malloc(sizeof(double) * (size_t)P1);
        double *px = (double *)malloc(sizeof(double) * (size_t)P1 * 3);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int64_t g = 0; g < ncell; ++g) {
            const int cx = centred((int)(g / ((int64_t)K * K)), K);
            const int cy = centred((int)((g / K) % K), K);
            const int cz = centred((int)(g % K), K);
            const int near = abs(cx) <= R && abs(cy) <= R && abs(cz) <= R;
            const double dx = cx * w, dy = cy * w, dz = cz * w;
            double *out = &D[g * nt];
            memset(out, 0, sizeof(double) * (size_t)nt);
            /* real space */
            for (int nx = -nimg; nx <= nimg; ++nx)
                for (int ny = -nimg; ny <= nimg; ++ny)
                    for (int nz = -nimg; nz <= nimg; ++nz) {
                        if (near && nx == 0 && ny == 0 && nz == 0) continue;
                        const double X = dx + nx * box, Y = dy + ny * box, Z = dz + nz * box;
                        const double r = sqrt(X * X + Y * Y + Z * Z);
                        if (r == 0.0) continue; /* only the excluded near image can sit at 0 */
                        gm_erfc(p, alpha, r, gm);
                        hermite_add(p, X, Y, Z, gm, 1.0, out, cur, nxt);
                    }
            /* reciprocal space */
            for (int64_t q = 0; q < nh; ++q) {
                if (kw[q] == 0.0) continue;
                const double kx = kv[3 * q], ky = kv[3 * q + 1], kz = kv[3 * q + 2];
                const double th = kx * dx + ky * dy + kz * dz;
                const double cs = cos(th), sn = sin(th);
                /* Re(i^s e^{i th}) for s mod 4 */
                const double val[4] = {cs, -sn, -cs, sn};
                for (int e = 0; e <= p; ++e) {
                    px[e] = e ? px[e - 1] * kx : 1.0;
                    px[P1 + e] = e ? px[P1 + e - 1] * ky : 1.0;
                    px[2 * P1 + e] = e ? px[2 * P1 + e - 1] * kz : 1.0;
                }
                int64_t t = 0;
                for (int a = 0; a <= p; ++a)
                    for (int b = 0; b <= p - a; ++b)
                        for (int c = 0; c <= p - a - b; ++c)
                            out[t++] += kw[q] * px[a] * px[P1 + b] * px[2 * P1 + c] * val[(a + b + c) & 3];
            }
            /* the constant of the neutralising background */
            out[0] += -M_PI / (alpha * alpha * V);
            /* remove the near image's smooth erf part */
            if (near) {
                gm_erf(p, alpha, sqrt(dx * dx + dy * dy + dz * dz), gm);
                hermite_add(p, dx, dy, dz, gm, -1.0, out, cur, nxt);
            }
        }
        free(cur);
        free(nxt);
        free(gm);
        free(px);
    }
    free(kw);
    free(kv);
    return 0;
}

/* Cartesian derivatives of 1/r at (X, Y, Z) != 0 for every term (a pin's
 * building block: the direct image sum converges for high orders). */
void oracle_coulomb_derivatives(int p, double X, double Y, double Z, double *out)
{
    const int P1 = p + 1;
    double *cur = (double *)malloc(sizeof(double) * (size_t)P1 * P1 * P1);
    double *nxt = (double *)malloc(sizeof(double) * (size_t)P1 * P1 * P1);
    double *gm = (double *)malloc(sizeof(double) * (size_t)P1);
    memset(out, 0, sizeof(double) * (size_t)nterms(p));
    gm_coulomb(p, sqrt(X * X + Y * Y + Z * Z), gm);
    hermite_add(p, X, Y, Z, gm, 1.0, out, cur, nxt);
    free(cur);
    free(nxt);
    free(gm);
}

/* Taylors by the direct cyclic convolution over cells (see the header). */
int oracle_convolve_direct(int K, int p, const double *D, const double *M, double *T)
{
    const int64_t nt = nterms(p);
    const int64_t ncell = (int64_t)K * K * K;
    double *fac = (double *)malloc(sizeof(double) * (size_t)(p + 1));
    for (int i = 0; i <= p; ++i) fac[i] = factorial(i);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t c = 0; c < ncell; ++c) {
        const int x = (int)(c / ((int64_t)K * K)), y = (int)((c / K) % K), z = (int)(c % K);
        double *out = &T[c * nt];
        memset(out, 0, sizeof(double) * (size_t)nt);
        for (int64_t s = 0; s < ncell; ++s) {
            const int sx = (int)(s / ((int64_t)K * K)), sy = (int)((s / K) % K), sz = (int)(s % K);
            const int64_t g = (((int64_t)((x - sx + K) % K) * K) + (y - sy + K) % K) * K + (z - sz + K) % K;
            const double *d = &D[g * nt];
            const double *m = &M[s * nt];
            for (int na = 0; na <= p; ++na)
                for (int nb = 0; nb <= p - na; ++nb)
                    for (int nc = 0; nc <= p - na - nb; ++nc) {
                        const int rem = p - na - nb - nc;
                        double acc = 0.0;
                        for (int ka = 0; ka <= rem; ++ka)
                            for (int kb = 0; kb <= rem - ka; ++kb)
                                for (int kc = 0; kc <= rem - ka - kb; ++kc) {
                                    const double sign = ((ka + kb + kc) & 1) ? -1.0 : 1.0;
                                    const double coef = sign / (fac[na] * fac[nb] * fac[nc] * fac[ka] * fac[kb] * fac[kc]);
                                    acc += coef * d[term_index(na + ka, nb + kb, nc + kc, p)] *
                                           m[term_index(ka, kb, kc, p)];
                                }
                        out[term_index(na, nb, nc, p)] += acc;
                    }
        }
    }
    free(fac);
    return 0;
}

/* a_i = sum_n T^n grad(x^n) (unit masses) for every particle, in input order;
 * x is the FP32 cell-centred offset times the cell width. */
int oracle_taylor_forces(const float *pos, int64_t N, double box, int K, int p, const double *T, double *out)
{
    const int64_t nt = nterms(p);
    const double kl = (double)K / box;
    const double w = box / (double)K;
    int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(| : bad)
#endif
    for (int64_t i = 0; i < N; ++i) {
        int cell[3];
        double x[3];
        for (int d = 0; d < 3; ++d) {
            float o = 0.0f;
            double wrap = 0.0;
            if (oracle_coord(pos[3 * i + d], kl, K, &cell[d], &o, &wrap)) bad = 1;
            x[d] = (double)o * w;
        }
        const double *t = &T[(((int64_t)cell[0] * K + cell[1]) * K + cell[2]) * nt];
        double ax = 0.0, ay = 0.0, az = 0.0;
        int64_t q = 0;
        for (int a = 0; a <= p; ++a)
            for (int b = 0; b <= p - a; ++b)
                for (int c = 0; c <= p - a - b; ++c, ++q) {
                    /* d/dx x^a y^b z^c = a x^(a-1) y^b z^c, and so on */
                    double xa = 1.0, yb = 1.0, zc = 1.0, xa1 = 0.0, yb1 = 0.0, zc1 = 0.0;
                    for (int e = 0; e < a; ++e) {
                        xa1 = (e == a - 1) ? xa : xa1;
                        xa *= x[0];
                    }
                    for (int e = 0; e < b; ++e) {
                        yb1 = (e == b - 1) ? yb : yb1;
                        yb *= x[1];
                    }
                    for (int e = 0; e < c; ++e) {
                        zc1 = (e == c - 1) ? zc : zc1;
                        zc *= x[2];
                    }
                    ax += t[q] * a * xa1 * yb * zc;
                    ay += t[q] * b * xa * yb1 * zc;
                    az += t[q] * c * xa * yb * zc1;
                }
        out[3 * i] = ax;
        out[3 * i + 1] = ay;
        out[3 * i + 2] = az;
    }
    return bad;
}

/* Ewald reference accelerations (unit masses) on the given sinks (all when
 * sinks is NULL): a_i = sum_{j != i} grad Phi(x_i - x_j). */
int oracle_ewald_forces(const float *pos, int64_t N, double box, double alpha, int nimg, int hmax,
                        const int64_t *sinks, int64_t nsinks, double *out)
{
    const double V = box * box * box;
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    for (int64_t i = 0; i < 3 * N; ++i) {
        const double v = (double)pos[i];
        if (!isfinite(v)) {
            free(x);
            return 1;
        }
        x[i] = v - box * floor(v / box);
    }
    const int H = 2 * hmax + 1;
    const int64_t nh = (int64_t)H * H * H;
    /* structure factors S(h) = sum_j exp(-i k.x_j) */
    double *Sre = (double *)calloc((size_t)nh, sizeof(double));
    double *Sim = (double *)calloc((size_t)nh, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8)
#endif
    for (int64_t q = 0; q < nh; ++q) {
        const int hx = (int)(q / (H * H)) - hmax, hy = (int)((q / H) % H) - hmax, hz = (int)(q % H) - hmax;
        if (hx == 0 && hy == 0 && hz == 0) continue;
        const double kx = 2.0 * M_PI * hx / box, ky = 2.0 * M_PI * hy / box, kz = 2.0 * M_PI * hz / box;
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            const double th = kx * x[3 * j] + ky * x[3 * j + 1] + kz * x[3 * j + 2];
            sr += cos(th);
            si -= sin(th);
        }
        Sre[q] = sr;
        Sim[q] = si;
    }
    const int64_t n = sinks ? nsinks : N;
    const double c2 = 2.0 * alpha / sqrt(M_PI);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t s = 0; s < n; ++s) {
        const int64_t i = sinks ? sinks[s] : s;
        double f[3] = {0.0, 0.0, 0.0};
        /* real space: grad erfc(alpha r)/r = -r_vec [erfc(alpha r)/r^3 + c2 exp(-alpha^2 r^2)/r^2] */
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double d0[3];
            for (int d = 0; d < 3; ++d) {
                double v = x[3 * i + d] - x[3 * j + d];
                v -= box * floor(v / box + 0.5);
                d0[d] = v;
            }
            for (int nx = -nimg; nx <= nimg; ++nx)
                for (int ny = -nimg; ny <= nimg; ++ny)
                    for (int nz = -nimg; nz <= nimg; ++nz) {
                        const double X = d0[0] + nx * box, Y = d0[1] + ny * box, Z = d0[2] + nz * box;
                        const double r2 = X * X + Y * Y + Z * Z;
                        const double r = sqrt(r2);
                        const double gfac = erfc(alpha * r) / (r2 * r) + c2 * exp(-alpha * alpha * r2) / r2;
                        f[0] -= gfac * X;
                        f[1] -= gfac * Y;
                        f[2] -= gfac * Z;
                    }
        }
        /* reciprocal space: -(4 pi/V) sum_h exp(-k^2/4alpha^2)/k^2 k Im[exp(i k.x_i) S(h)] */
        for (int64_t q = 0; q < nh; ++q) {
            const int hx = (int)(q / (H * H)) - hmax, hy = (int)((q / H) % H) - hmax, hz = (int)(q % H) - hmax;
            if (hx == 0 && hy == 0 && hz == 0) continue;
            const double kx = 2.0 * M_PI * hx / box, ky = 2.0 * M_PI * hy / box, kz = 2.0 * M_PI * hz / box;
            const double k2 = kx * kx + ky * ky + kz * kz;
            const double wk = (4.0 * M_PI / V) * exp(-k2 / (4.0 * alpha * alpha)) / k2;
            const double th = kx * x[3 * i] + ky * x[3 * i + 1] + kz * x[3 * i + 2];
            const double im = sin(th) * Sre[q] + cos(th) * Sim[q];
            f[0] -= wk * kx * im;
            f[1] -= wk * ky * im;
            f[2] -= wk * kz * im;
        }
        out[3 * s] = f[0];
        out[3 * s + 1] = f[1];
        out[3 * s + 2] = f[2];
    }
    free(x);
    free(Sre);
    free(Sim);
    return 0;
}
