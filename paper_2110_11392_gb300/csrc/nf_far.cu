// Far field of the force split (Sec. "Far-field Computation"): the
// derivatives tensor, the convolution of the cell multipoles with it on the
// K^3 grid (by FFT), and the acceleration from the resulting Taylor series.
//
// Derivatives tensor.  D^{abc}(g), for every cell offset g (sink minus source
// cell, mod K), is the (a,b,c)-th Cartesian derivative of the periodic
// potential of a unit mass at the cell-centre separation: every image of the
// box, the images of the central and near-field cells included, with the
// uniform neutralising background of Ewald summation, minus the single image
// that the near field computes directly (an offset whose centred components
// all lie in [-R, R]).  With Ewald's split at parameter alpha
//     sum_n 1/|r+nL| = sum_n erfc(alpha|r+nL|)/|r+nL|
//                      + (4 pi / V) sum_{k != 0} exp(-k^2 / 4 alpha^2) / k^2 cos(k.r)
//                      - pi / (alpha^2 V),                k = 2 pi h / L,
// the real-space images are summed on the grid (k_deriv_real) and the
// reciprocal part is added after the FFT directly in k-space: on the grid
// r = g w, its discrete Fourier transform at q is K^3 times the sum of
// (4 pi/V) exp(-k^2/4alpha^2)/k^2 (i k)^{abc} over the h congruent to q mod K
// (k_deriv_recip), so it needs no real-space evaluation at all.
// Cartesian derivatives of a radial g(r) use the Hermite recursion of
// McMurchie & Davidson (1978): with g_m = (r^-1 d/dr)^m g and R^m_{tuv} the
// (t,u,v) derivative of g_m, R^m_{t+1,u,v} = t R^{m+1}_{t-1,u,v} +
// X R^{m+1}_{t,u,v} (likewise in Y, Z) and R^0_{abc} is the derivative.  For
// erfc(alpha r)/r, g_m = (-1)^m B_m with B_0 = erfc(alpha r)/r and
// B_m = [(2m-1) B_{m-1} + (2 alpha^2)^m exp(-alpha^2 r^2) / (alpha sqrt(pi))] / r^2
// (Smith's recurrence).  The near image's smooth erf(alpha r)/r part is
// subtracted with g_m from its power series (alpha r < 2) or as the Coulomb
// g_m minus the erfc g_m (alpha r >= 2, where that difference is well
// conditioned).
//
// Taylors.  T^n(c) = sum_{c'} sum_k (-1)^{|k|} / (n! k!) D^{n+k}(c - c') M^k(c'),
// |n| + |k| <= p: the Taylor expansion of 1/|Delta + x - s| in the sink and
// source displacements about the cell-centre separation.  By the convolution
// theorem each term is a product in k-space (k_far_contract) between the
// forward transforms of D and of the multipoles; the inverse transform gives
// T in every cell.  The convolution runs on the (p+1)^2 reduced terms (see
// far_tables) and the complete Taylors are rebuilt per cell
// (k_far_rebuild).  The transforms are this file's kernels: radix-4/2 ones
// in double-float for a power-of-two K (k_fft_*), mixed-radix ones for any K
// in double-float or FP64 (k_gfft_*); every step is a kernel of this file.  The per-particle work runs in cell units
// (multipoles of the stored offsets x / w, Taylors T'^n = T^n w^{|n|}); the
// factors w^{|n|+|k|} live in the convolution's coefficients.
//
// Acceleration.  The potential in a cell is -m sum_n T^n x^n (G = 1), so
// a = m sum_n T^n grad(x^n) = (m / w) sum_n T'^n grad'(x'^n), x' the
// particle's FP32 cell-centred offset, evaluated by nested Horner schemes in
// z, y and x (k_taylor_forces).  The derivatives are FP64.  The rest is
// FP64 (k_multipoles in nf_multipole.cu, k_far_reduce, k_gfft_*,
// k_far_contract, k_taylor_forces) or double-float on the FP32 pipe
// (k_multipoles_red_df, k_fft_* or k_gfft_*, k_far_contract_df,
// k_taylor_forces_df), as the caller selects.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "nf_internal.cuh"

namespace nf {

namespace {

constexpr int kDerivThreads = 256;

__host__ __device__ constexpr int far_terms(int p) { return (p + 3) * (p + 2) * (p + 1) / 6; }

// (a, b, c) of term t in the complete-basis order of order p
__device__ inline void decode_term(int t, int p, int& a, int& b, int& c)
{
    int r = t;
    for (a = 0; a <= p; ++a) {
        const int n_a = (p - a + 1) * (p - a + 2) / 2;
        if (r < n_a) break;
        r -= n_a;
    }
    for (b = 0; b <= p - a; ++b) {
        const int n_b = p - a - b + 1;
        if (r < n_b) break;
        r -= n_b;
    }
    c = r;
}

__host__ __device__ inline int encode_term(int a, int b, int c, int p)
{
    int t = 0;
    for (int a2 = 0; a2 < a; ++a2) t += (p - a2 + 1) * (p - a2 + 2) / 2;
    for (int b2 = 0; b2 < b; ++b2) t += p - a - b2 + 1;
    return t + c;
}

__device__ inline int centred(int g, int K) { return 2 * g > K ? g - K : g; }

// g_m of erfc(alpha r)/r (sign (-1)^m included), m = 0..p
__device__ void gm_erfc(int p, double alpha, double r, double* gm)
{
    const double r2 = r * r;
    const double e = exp(-alpha * alpha * r2) / (alpha * 1.7724538509055160273);
    double B = erfc(alpha * r) / r, pw = 1.0;
    gm[0] = B;
    for (int m = 1; m <= p; ++m) {
        pw *= 2.0 * alpha * alpha;
        B = ((2 * m - 1) * B + pw * e) / r2;
        gm[m] = (m & 1) ? -B : B;
    }
}

// g_m of erf(alpha r)/r, m = 0..p, any r >= 0
__device__ void gm_erf(int p, double alpha, double r, double* gm)
{
    if (alpha * r >= 2.0) {
        gm_erfc(p, alpha, r, gm);
        double v = 1.0 / r;
        const double ir2 = 1.0 / (r * r);
        for (int m = 0; m <= p; ++m) {
            if (m) v *= -(double)(2 * m - 1) * ir2;
            gm[m] = v - gm[m];
        }
        return;
    }
    const double x = -r * r;
    double am = alpha;  // alpha^(2m+1)
    double sgn = 1.0;   // (-2)^m
    for (int m = 0; m <= p; ++m) {
        double sum = 0.0, term = 1.0, ap = am;
        for (int j = 0; j < 120; ++j) {
            const double add = term * ap / (double)(2 * m + 2 * j + 1);
            sum += add;
            if (j > 4 && fabs(add) <= 1e-18 * fabs(sum)) break;
            term *= x / (double)(j + 1);
            ap *= alpha * alpha;
        }
        gm[m] = 1.1283791670955125739 * sgn * sum;  // 2/sqrt(pi)
        am *= alpha * alpha;
        sgn *= -2.0;
    }
}

// Hermite recursion of one warp for one point: adds scale * R^0_{abc} of the
// point to the warp's accumulators acc[nt] (shared memory).  The layers are
// compact: the entry of (t, u, v) is its term index in the order-p basis
// (enc maps (t, u, v) to it, dec back), so two layers take 2 nt doubles;
// gm holds the p + 1 values g_m at the point.
__device__ void hermite_warp(int p, int nt, double X, double Y, double Z, const double* gm, double scale,
                             double* lay0, double* lay1, const short* enc, const char4* dec, double* acc)
{
    const int lane = threadIdx.x & 31;
    const int P1 = p + 1;
    double* nxt = lay0;
    double* cur = lay1;
    if (lane == 0) nxt[0] = gm[p];  // layer p holds only (0, 0, 0), term 0
    __syncwarp();
    for (int m = p - 1; m >= 0; --m) {
        const int top = p - m;
        for (int e = lane; e < nt; e += 32) {
            const char4 d = dec[e];
            const int t = d.x, u = d.y, v = d.z;
            if (t + u + v > top) continue;
            double r;
            if (t + u + v == 0)
                r = gm[m];
            else if (t > 0)
                r = (t >= 2 ? (t - 1) * nxt[enc[((t - 2) * P1 + u) * P1 + v]] : 0.0) +
                    X * nxt[enc[((t - 1) * P1 + u) * P1 + v]];
            else if (u > 0)
                r = (u >= 2 ? (u - 1) * nxt[enc[(t * P1 + u - 2) * P1 + v]] : 0.0) +
                    Y * nxt[enc[(t * P1 + u - 1) * P1 + v]];
            else
                r = (v >= 2 ? (v - 1) * nxt[enc[(t * P1 + u) * P1 + v - 2]] : 0.0) +
                    Z * nxt[enc[(t * P1 + u) * P1 + v - 1]];
            cur[e] = r;
        }
        __syncwarp();
        double* sw = cur;
        cur = nxt;
        nxt = sw;
    }
    // layer 0 (every term) is in nxt
    for (int e = lane; e < nt; e += 32) acc[e] += scale * nxt[e];
    __syncwarp();
}

constexpr int kDerivWarps = kDerivThreads / 32;

size_t deriv_real_smem(int p)
{
    const int nt = far_terms(p), P1 = p + 1;
    const size_t doubles = (size_t)kDerivWarps * (3 * nt + P1);  // accumulators, two layers, g_m per warp
    const size_t shorts = (size_t)((P1 * P1 * P1 + 1) & ~1);
    return doubles * sizeof(double) + shorts * sizeof(short) + (size_t)nt * sizeof(char4);
}

// Real-space part of D, one block per cell offset g: images n in [-nimg, nimg]^3
// (the near image left out), minus the near image's erf part.  Each warp
// takes its own images (one Hermite recursion per image, layers private to the
// warp); the warps' sums are added in a fixed order at the end.  D is
// cell-major [C][nt], the layout of the multipoles.
__global__ void __launch_bounds__(kDerivThreads) k_deriv_real(int K, int R, int p, int nt, double box, double alpha,
                                                              int nimg, double* __restrict__ D)
{
    extern __shared__ double sm[];
    const int P1 = p + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* acc_all = sm;                                  // [warps][nt]
    double* lay_all = acc_all + (size_t)kDerivWarps * nt;  // [warps][2][nt]
    double* gm_all = lay_all + (size_t)kDerivWarps * 2 * nt;  // [warps][P1]
    short* enc = reinterpret_cast<short*>(gm_all + (size_t)kDerivWarps * P1);
    char4* dec = reinterpret_cast<char4*>(enc + ((P1 * P1 * P1 + 1) & ~1));
    for (int e = threadIdx.x; e < nt; e += blockDim.x) {
        int a, b, c;
        decode_term(e, p, a, b, c);
        dec[e] = make_char4((char)a, (char)b, (char)c, 0);
        enc[(a * P1 + b) * P1 + c] = (short)e;
    }
    __syncthreads();  // the tables are read by every warp
    double* acc = acc_all + (size_t)warp * nt;
    double* lay0 = lay_all + (size_t)warp * 2 * nt;
    double* lay1 = lay0 + nt;
    double* gm = gm_all + (size_t)warp * P1;
    const int C = K * K * K;
    const double w = box / K;
    const int side = 2 * nimg + 1, nimages = side * side * side;
    for (int g = blockIdx.x; g < C; g += gridDim.x) {
        const int cx = centred(g / (K * K), K), cy = centred((g / K) % K, K), cz = centred(g % K, K);
        const bool near = abs(cx) <= R && abs(cy) <= R && abs(cz) <= R;
        const double dx = cx * w, dy = cy * w, dz = cz * w;
        for (int e = lane; e < nt; e += 32) acc[e] = 0.0;
        __syncwarp();
        // images 0 .. nimages-1, and for a near offset one more item: its erf part
        for (int n = warp; n < nimages + (near ? 1 : 0); n += kDerivWarps) {
            double X = dx, Y = dy, Z = dz, scale = -1.0;
            if (n < nimages) {
                const int nx = n / (side * side) - nimg, ny = (n / side) % side - nimg, nz = n % side - nimg;
                if (near && nx == 0 && ny == 0 && nz == 0) continue;
                X = dx + nx * box;
                Y = dy + ny * box;
                Z = dz + nz * box;
                scale = 1.0;
                if (lane == 0) gm_erfc(p, alpha, sqrt(X * X + Y * Y + Z * Z), gm);
            } else if (lane == 0) {
                gm_erf(p, alpha, sqrt(dx * dx + dy * dy + dz * dz), gm);
            }
            __syncwarp();
            hermite_warp(p, nt, X, Y, Z, gm, scale, lay0, lay1, enc, dec, acc);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nt; t += blockDim.x) {
            double sum = 0.0;
            for (int q = 0; q < kDerivWarps; ++q) sum += acc_all[(size_t)q * nt + t];
            D[(size_t)g * nt + t] = sum;
        }
        __syncthreads();
    }
}

// Reciprocal part and background constant, added to the transformed real-space
// part, and the result compressed to one real number per (term, q).
// Dh (input) is the transform of the real-space part, [nt][K][K][K/2+1];
// the reciprocal part adds K^3 sum_{h = q mod K, h != 0, |h_i| <= hmax}
// w(k) (i k)^{abc}.  D^{abc}(-g) = (-1)^{a+b+c} D^{abc}(g) on the periodic
// grid, so the transform of a term is real for even a+b+c and imaginary for
// odd a+b+c (the parity the paper uses to halve the convolution): Dr keeps
// the real part of even terms and the imaginary part of odd ones.
__global__ void k_deriv_recip(int K, int p, int nt, double box, double alpha, int hmax,
                              const double2* __restrict__ Dh, double* __restrict__ Dr)
{
    const int KH = K / 2 + 1;
    const long long nq = (long long)K * K * KH;
    const long long total = nq * nt;
    const double V = box * box * box;
    const double twopi_L = 6.283185307179586477 / box;
    const double K3 = (double)K * K * K;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(e / nq);
        const long long q = e - (long long)t * nq;
        const int qx = (int)(q / (K * KH)), qy = (int)((q / KH) % K), qz = (int)(q % KH);
        int a, b, c;
        decode_term(t, p, a, b, c);
        const int s = a + b + c;
        double acc = 0.0;  // coefficient of i^(s mod 2): real part (s even) or imaginary part (s odd)
        for (int hx = -hmax + (qx + hmax) % K; hx <= hmax; hx += K)
            for (int hy = -hmax + (qy + hmax) % K; hy <= hmax; hy += K)
                for (int hz = -hmax + (qz + hmax) % K; hz <= hmax; hz += K) {
                    if (hx == 0 && hy == 0 && hz == 0) continue;
                    const double kx = twopi_L * hx, ky = twopi_L * hy, kz = twopi_L * hz;
                    const double k2 = kx * kx + ky * ky + kz * kz;
                    double f = (12.566370614359172954 / V) * exp(-k2 / (4.0 * alpha * alpha)) / k2;
                    for (int i = 0; i < a; ++i) f *= kx;
                    for (int i = 0; i < b; ++i) f *= ky;
                    for (int i = 0; i < c; ++i) f *= kz;
                    // i^s = +1, +i, -1, -i for s mod 4 = 0, 1, 2, 3
                    acc += (s & 2) ? -f : f;
                }
        const double2 v = Dh[e];
        double out = ((s & 1) ? v.y : v.x) + K3 * acc;
        if (t == 0 && q == 0) out += K3 * (-3.14159265358979323846 / (alpha * alpha * V));
        Dr[e] = out;
    }
}

// Th[n][q] = scale * sum_{pairs of n} coef * D^{n+k}(q) * Mh[k][q], one thread
// per (n, q), q fastest: a warp shares n, so the pair list is a broadcast and
// the Dr and Mh rows are read coalesced; one thread per q alone would leave
// a few warps per SM waiting on their dependent FMA chains.  D^{j}(q) is
// Dr[j][q] for even |j| and i Dr[j][q] for odd |j|, so a pair costs one
// real-times-complex product (3 FP64 operations) instead of a complex one.
__global__ void __launch_bounds__(256) k_far_contract(long long nq, int nt, const int* __restrict__ seg,
                                                      const FarPair* __restrict__ pairs,
                                                      const double* __restrict__ Dr,
                                                      const double2* __restrict__ Mh, double2* __restrict__ Th,
                                                      double scale)
{
    const long long total = nq * nt;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(e / nq);
        const long long q = e - (long long)n * nq;
        double re = 0.0, im = 0.0;
        const int e1 = seg[n + 1];
        for (int i = seg[n]; i < e1; ++i) {
            const FarPair pr = pairs[i];
            const double cd = pr.coef * Dr[(size_t)(pr.j & 0x7fffffff) * nq + q];
            const double2 m = Mh[(size_t)pr.k * nq + q];
            // odd |j|: i * cd * m = (-cd m.y, cd m.x).  The rotation is done with
            // integer selects and a sign-bit flip, so the FP64 pipe sees exactly
            // one multiply and two FMAs per pair.
            const bool odd = pr.j < 0;
            const double mr = odd ? m.y : m.x, mi = odd ? m.x : m.y;
            const double cr = __longlong_as_double(__double_as_longlong(cd) ^ (odd ? (long long)0x8000000000000000ull : 0ll));
            re = fma(cr, mr, re);
            im = fma(cd, mi, im);
        }
        Th[e] = make_double2(scale * re, scale * im);
    }
}

// Far-field acceleration of every particle, one thread per particle in the
// binned order; the particle's cell comes from a binary search of the cell
// offsets (cells are ragged, so one block per cell would leave most of a
// block idle).  The potential sum_{a,b,c} T_{abc} x^a y^b z^c and its
// gradient are evaluated by nested Horner schemes (in z, then y, then x),
// each carrying its derivative along: no power tables, about two FMAs per
// term.  a = m * gradient.  Writes acc_far[orig] (FP64) and/or adds to
// acc_add[orig] (FP32).
template <int P>
__global__ void __launch_bounds__(128) k_taylor_forces(const int* __restrict__ off, const float4* __restrict__ rel,
                                                      const double* __restrict__ T, int N, int C, double w,
                                                      double mass, double* __restrict__ acc_far,
                                                      float* __restrict__ acc_add)
{
    constexpr int NT = (P + 3) * (P + 2) * (P + 1) / 6;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        // the cell with off[cell] <= i < off[cell + 1]
        int lo = 0, hi = C;  // off[lo] <= i < off[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(off + mid) <= i)
                lo = mid;
            else
                hi = mid;
        }
        const double* __restrict__ Tc = T + (size_t)lo * NT;
        const float4 r4 = rel[i];
        const double x = (double)r4.x * w, y = (double)r4.y * w, z = (double)r4.z * w;
        double F = 0.0, Fx = 0.0, Fy = 0.0, Fz = 0.0;
        // rolled loops: FP64 arithmetic, not issue, is the limit, and full
        // unrolling would hoist every coefficient load into registers
#pragma unroll 1
        for (int a = P; a >= 0; --a) {
            // terms with first index a start at NT - C(P - a + 3, 3)
            const int base_a = NT - (P - a + 3) * (P - a + 2) * (P - a + 1) / 6;
            double U = 0.0, Uy = 0.0, Uz = 0.0;
#pragma unroll 1
            for (int b = P - a; b >= 0; --b) {
                const int base = base_a + b * (P - a + 1) - b * (b - 1) / 2;
                double S = 0.0, Sz = 0.0;
                for (int c = P - a - b; c >= 0; --c) {
                    Sz = fma(Sz, z, S);
                    S = fma(S, z, __ldg(Tc + base + c));
                }
                Uy = fma(Uy, y, U);
                U = fma(U, y, S);
                Uz = fma(Uz, y, Sz);
            }
            Fx = fma(Fx, x, F);
            F = fma(F, x, U);
            Fy = fma(Fy, x, Uy);
            Fz = fma(Fz, x, Uz);
        }
        const int orig = __float_as_int(r4.w);
        const double ax = mass * Fx, ay = mass * Fy, az = mass * Fz;
        if (acc_far) {
            acc_far[3 * (size_t)orig] = ax;
            acc_far[3 * (size_t)orig + 1] = ay;
            acc_far[3 * (size_t)orig + 2] = az;
        }
        if (acc_add) {
            acc_add[3 * (size_t)orig] += (float)ax;
            acc_add[3 * (size_t)orig + 1] += (float)ay;
            acc_add[3 * (size_t)orig + 2] += (float)az;
        }
    }
}

// ---- double-float arithmetic ------------------------------------------------
// GB300 runs FP64 at 1/64 of the FP32 rate.  The per-particle far-field
// kernels therefore also exist in double-float form: a value is an unevaluated
// sum hi + lo of two FP32 numbers, kept exact by the error-free
// transformations TwoSum (Knuth), FastTwoSum (Dekker) and TwoProduct by FMA
// (Ogita, Rump & Oishi 2005), which carry about 48 significant bits on the
// FP32 pipe.  The _rn intrinsics keep the compiler from fusing a product into
// a following sum, which would break the exactness of the transformations.
struct __align__(8) dfl {
    float h, l;
};

__device__ __forceinline__ dfl df_fast(float a, float b)  // |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// a * z + t for a float z, without the final renormalisation: the result is
// the unevaluated sum of TwoSum's high part and the collected error terms,
// which a following step takes as it is (its exact product and TwoSum need
// no normalised input).  Used inside Horner chains, where it saves three of
// fourteen instructions per step.
__device__ __forceinline__ dfl df_fma_f_nr(dfl a, float z, dfl t)
{
    const float p = __fmul_rn(a.h, z);
    float e = __fmaf_rn(a.h, z, -p);
    e = __fmaf_rn(a.l, z, e);
    const dfl s = df_two_sum(p, t.h);
    return {s.h, __fadd_rn(s.l, __fadd_rn(e, t.l))};
}

// a * b + t without the final renormalisation (see df_fma_f_nr)
__device__ __forceinline__ dfl df_fma_nr(dfl a, dfl b, dfl t)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const dfl s = df_two_sum(p, t.h);
    return {s.h, __fadd_rn(s.l, __fadd_rn(e, t.l))};
}

// a * b + t
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl t)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const dfl s = df_two_sum(p, t.h);
    return df_fast(s.h, __fadd_rn(s.l, __fadd_rn(e, t.l)));
}

__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_fast(p, e);
}

// a * z for a float z
__device__ __forceinline__ dfl df_mul_f(dfl a, float z)
{
    const float p = __fmul_rn(a.h, z);
    float e = __fmaf_rn(a.h, z, -p);
    e = __fmaf_rn(a.l, z, e);
    return df_fast(p, e);
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    const dfl s = df_two_sum(a.h, b.h);
    return df_fast(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ dfl df_from(double v)
{
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}

// ---- double-float transforms and k-space product ---------------------------
// GB300's FP64 pipe makes double-precision transforms and the FP64 k-space
// product the slow part of the convolution.  In double-float mode they run on
// the FP32 pipe instead (for a power-of-two K with these kernels, otherwise
// with the mixed-radix ones below): a complex value is a
// float4 {re.h, re.l, im.h, im.l}.  The 3-D real transform is three passes of
// 1-D transforms over lines held in shared memory (bit-reversed on load,
// pairs of radix-2 stages done as one radix-4 step with one __syncthreads,
// twiddles e^{-2 pi i j/K} as double-float pairs built on the host from FP64
// cos/sin).  Layouts: the real
// side is cell-major [x][y][z][field], the spectrum term-major
// [field][x][y][kz] with kz in 0..K/2; forward is e^{-i...}, the inverse is
// unnormalised (the 1/K^3 sits in the k-space product).
struct cdf {
    dfl re, im;
};
__device__ __forceinline__ cdf cdf_ld(float4 v) { return {dfl{v.x, v.y}, dfl{v.z, v.w}}; }
__device__ __forceinline__ float4 cdf_st(cdf v) { return make_float4(v.re.h, v.re.l, v.im.h, v.im.l); }
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dfl df_half(dfl a) { return {0.5f * a.h, 0.5f * a.l}; }  // exact
__device__ __forceinline__ cdf cdf_mul(cdf w, cdf x)
{
    return {df_fma(w.re, x.re, df_neg(df_mul(w.im, x.im))), df_fma(w.re, x.im, df_mul(w.im, x.re))};
}
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) { return {df_add(a.re, df_neg(b.re)), df_add(a.im, df_neg(b.im))}; }

constexpr int kFftThreads = 256;
constexpr int kFftPoints = 2048;  // complex points of one block's lines in shared memory

__host__ __device__ inline int fft_lines_per_block(int K) { return K >= kFftPoints ? 1 : kFftPoints / K; }
// The z passes transform lines of K/2 points: twice as many lines fit.
__host__ __device__ inline int fft_z_lines_per_block(int K) { return fft_lines_per_block(K / 2); }

// The stages over nl lines of K points in shared memory (bit-reversed order
// in, natural order out), two radix-2 stages at a time: a thread loads four
// points i0 + {0, h, 2h, 3h}, applies stage h (twiddle W_2h^pos on both
// pairs) and stage 2h (W_4h^pos, and W_4h^{pos+h} = W_4h^pos * (-i)), and
// stores them; a last radix-2 stage when log2 K is odd.  tw: a table of
// e^{-2 pi i j / (K 2^tws)}, j < K 2^tws / 2 (tws = 1: a K-point transform
// using the table of twice its length); INV uses the conjugates (and +i).
__device__ __forceinline__ cdf cdf_tw(const float4* tw, int j, bool inv)
{
    float4 w4 = tw[j];
    if (inv) {
        w4.z = -w4.z;
        w4.w = -w4.w;
    }
    return cdf_ld(w4);
}

template <bool INV>
__device__ __forceinline__ void fft_stages(float4* line, int nl, int K, int logK, const float4* tw, int tws)
{
    int lh = 0;
    for (; lh + 1 < logK; lh += 2) {
        const int h = 1 << lh, s1 = logK - 1 - lh + tws, s2 = logK - 2 - lh + tws;
        const int quarter = K >> 2;
        for (int b = threadIdx.x; b < nl * quarter; b += blockDim.x) {
            const int l = b >> (logK - 2), j = b & (quarter - 1);
            const int pos = j & (h - 1);
            const int i0 = ((j - pos) << 2) + pos;
            float4* L = line + (size_t)l * K;
            const cdf x0 = cdf_ld(L[i0]), x1 = cdf_ld(L[i0 + h]), x2 = cdf_ld(L[i0 + 2 * h]), x3 = cdf_ld(L[i0 + 3 * h]);
            const cdf w1 = cdf_tw(tw, pos << s1, INV), w2 = cdf_tw(tw, pos << s2, INV);
            const cdf t1 = cdf_mul(w1, x1), t3 = cdf_mul(w1, x3);
            const cdf a0 = cdf_add(x0, t1), a1 = cdf_sub(x0, t1), a2 = cdf_add(x2, t3), a3 = cdf_sub(x2, t3);
            const cdf u2 = cdf_mul(w2, a2);
            const cdf v = cdf_mul(w2, a3);
            // times -i (forward) or +i (inverse)
            const cdf u3 = INV ? cdf{df_neg(v.im), v.re} : cdf{v.im, df_neg(v.re)};
            L[i0] = cdf_st(cdf_add(a0, u2));
            L[i0 + 2 * h] = cdf_st(cdf_sub(a0, u2));
            L[i0 + h] = cdf_st(cdf_add(a1, u3));
            L[i0 + 3 * h] = cdf_st(cdf_sub(a1, u3));
        }
        __syncthreads();
    }
    if (lh < logK) {  // the last stage, radix 2
        const int h = 1 << lh, sh = logK - 1 - lh + tws;
        const int half = K >> 1;
        for (int b = threadIdx.x; b < nl * half; b += blockDim.x) {
            const int l = b >> (logK - 1), j = b & (half - 1);
            const int pos = j & (h - 1);
            const int i0 = ((j - pos) << 1) + pos, i1 = i0 + h;
            float4* L = line + (size_t)l * K;
            const cdf u = cdf_ld(L[i0]);
            const cdf t = cdf_mul(cdf_tw(tw, pos << sh, INV), cdf_ld(L[i1]));
            L[i0] = cdf_st(cdf_add(u, t));
            L[i1] = cdf_st(cdf_sub(u, t));
        }
        __syncthreads();
    }
}

// x / d for a block-invariant d by a multiply-high with m = ceil(2^32 / d):
// exact for x < 2^32 / d (here x < 2^20, d <= 2^11).
struct FastDiv {
    unsigned long long m;
    int d;
    __device__ explicit FastDiv(int dv) : m(((1ull << 32) + (unsigned long long)dv - 1) / (unsigned long long)dv), d(dv) {}
    __device__ __forceinline__ int div(int x) const { return (int)(((unsigned long long)(unsigned)x * m) >> 32); }
};

__device__ __forceinline__ int fft_rev(int i, int logK) { return logK ? (int)(__brev((unsigned)i) >> (32 - logK)) : 0; }

// Forward z pass: real double-float fields, cell-major [x][y][z][nf], to the
// spectrum S [nf][x][y][kz].  Block: one (x, y) and a chunk of fields.  Each
// real line of K points is transformed as a complex line of M = K/2 points,
// z[m] = x[2m] + i x[2m+1] (same line, so no mixing of fields of different
// size); with Z its transform, the even- and odd-sample transforms are
// E = (Z[k] + conj Z[M-k]) / 2 and O = (Z[k] - conj Z[M-k]) / 2i, and
// X[k] = E[k] + W^k O[k], W = e^{-2 pi i/K}, for k = 0..M.
__global__ void __launch_bounds__(kFftThreads) k_fft_z_fwd(const dfl* __restrict__ R, int K, int logK, int nf,
                                                           int nchunk, const float4* __restrict__ twg,
                                                           float4* __restrict__ S)
{
    extern __shared__ float4 fsm[];
    float4* tw = fsm;
    float4* line = fsm + K / 2;
    const int M = K / 2, logM = logK - 1, H = M + 1;
    const int FB = fft_z_lines_per_block(K);
    const int chunk = blockIdx.x % nchunk;
    const long long xy = blockIdx.x / nchunk;
    const int f0 = chunk * FB, nfc = min(FB, nf - f0);
    for (int j = threadIdx.x; j < M; j += blockDim.x) tw[j] = twg[j];
    const dfl* src = R + (size_t)xy * K * nf + f0;
    float2* halves = reinterpret_cast<float2*>(line);  // a point's real pair, then its imaginary pair
    const FastDiv by_nfc(nfc), by_H(H);
    for (int idx = threadIdx.x; idx < K * nfc; idx += blockDim.x) {
        const int z = by_nfc.div(idx), fl = idx - z * nfc;
        const dfl v = src[(size_t)z * nf + fl];
        halves[2 * ((size_t)fl * M + fft_rev(z >> 1, logM)) + (z & 1)] = make_float2(v.h, v.l);
    }
    __syncthreads();
    fft_stages<false>(line, nfc, M, logM, tw, 1);
    const size_t fstride = (size_t)K * K * H;
    for (int idx = threadIdx.x; idx < nfc * H; idx += blockDim.x) {
        const int fl = by_H.div(idx), k = idx - fl * H;
        const float4* L = line + (size_t)fl * M;
        const cdf a = cdf_ld(L[k & (M - 1)]), b = cdf_ld(L[(M - k) & (M - 1)]);
        const cdf e = {df_half(df_add(a.re, b.re)), df_half(df_add(a.im, df_neg(b.im)))};
        const cdf o = {df_half(df_add(a.im, b.im)), df_half(df_add(b.re, df_neg(a.re)))};
        const cdf x = k < M ? cdf_add(e, cdf_mul(cdf_ld(tw[k]), o)) : cdf_sub(e, o);  // W^M = -1
        S[(size_t)(f0 + fl) * fstride + (size_t)xy * H + k] = cdf_st(x);
    }
}

// Complex passes along y or x, in place on the spectrum S [nf][x][y][kz]:
// lines of K points at stride pstride, W consecutive kz per block.  Block:
// one (field, other index, kz chunk).
template <bool INV>
__global__ void __launch_bounds__(kFftThreads) k_fft_lines(float4* __restrict__ S, int K, int logK, int nA,
                                                           long long astride, long long pstride, int nchunk,
                                                           const float4* __restrict__ twg)
{
    extern __shared__ float4 fsm[];
    float4* tw = fsm;
    float4* line = fsm + K / 2;
    const int H = K / 2 + 1;
    const int W = fft_lines_per_block(K);
    const int chunk = blockIdx.x % nchunk;
    const long long fa = blockIdx.x / nchunk;
    const long long f = fa / nA, a = fa - f * nA;
    const int k0 = chunk * W, wc = min(W, H - k0);
    for (int j = threadIdx.x; j < K / 2; j += blockDim.x) tw[j] = twg[j];
    float4* base = S + f * (long long)K * K * H + a * astride + k0;
    const FastDiv by_wc(wc);
    for (int idx = threadIdx.x; idx < K * wc; idx += blockDim.x) {
        const int pt = by_wc.div(idx), w = idx - pt * wc;
        line[(size_t)w * K + fft_rev(pt, logK)] = base[pt * pstride + w];
    }
    __syncthreads();
    fft_stages<INV>(line, wc, K, logK, tw, 0);
    for (int idx = threadIdx.x; idx < K * wc; idx += blockDim.x) {
        const int pt = by_wc.div(idx), w = idx - pt * wc;
        base[pt * pstride + w] = line[(size_t)w * K + pt];
    }
}

// Inverse z pass: spectrum S [nf][x][y][kz] (kz <= K/2, the rest by Hermitian
// symmetry) to real double-float fields, cell-major [x][y][z][nf], through a
// complex transform of M = K/2 points: with X[k+M] = conj X[M-k],
// A = X[k] + X[k+M] and B = (X[k] - X[k+M]) W^{-k} are the transforms of the
// even and odd samples, and the inverse of Z = A + i B is x[2m] + i x[2m+1]
// (unnormalised, like the K-point inverse).  The imaginary parts at kz = 0
// and K/2 are ignored, as a complex-to-real transform does.
__global__ void __launch_bounds__(kFftThreads) k_fft_z_inv(const float4* __restrict__ S, int K, int logK, int nf,
                                                           int nchunk, const float4* __restrict__ twg,
                                                           dfl* __restrict__ R)
{
    extern __shared__ float4 fsm[];
    float4* tw = fsm;
    float4* line = fsm + K / 2;
    const int M = K / 2, logM = logK - 1, H = M + 1;
    const int FB = fft_z_lines_per_block(K);
    const int chunk = blockIdx.x % nchunk;
    const long long xy = blockIdx.x / nchunk;
    const int f0 = chunk * FB, nfc = min(FB, nf - f0);
    for (int j = threadIdx.x; j < M; j += blockDim.x) tw[j] = twg[j];
    __syncthreads();  // the pre-processing below reads the twiddles
    const size_t fstride = (size_t)K * K * H;
    for (int idx = threadIdx.x; idx < nfc * M; idx += blockDim.x) {
        const int fl = idx >> logM, k = idx - (fl << logM);
        const float4* row = S + (size_t)(f0 + fl) * fstride + (size_t)xy * H;
        float4 xk = row[k], xm = row[M - k];
        if (k == 0) {
            xk.z = xk.w = 0.0f;
            xm.z = xm.w = 0.0f;
        }
        const cdf a = cdf_ld(xk);
        const cdf bc = {dfl{xm.x, xm.y}, dfl{-xm.z, -xm.w}};  // X[k+M] = conj X[M-k]
        const cdf sum = cdf_add(a, bc), dif = cdf_sub(a, bc);
        float4 w4 = tw[k];
        w4.z = -w4.z;
        w4.w = -w4.w;
        const cdf bb = cdf_mul(cdf_ld(w4), dif);
        const cdf zz = {df_add(sum.re, df_neg(bb.im)), df_add(sum.im, bb.re)};
        line[(size_t)fl * M + fft_rev(k, logM)] = cdf_st(zz);
    }
    __syncthreads();
    fft_stages<true>(line, nfc, M, logM, tw, 1);
    dfl* dst = R + (size_t)xy * K * nf + f0;
    const FastDiv by_nfc(nfc);
    for (int idx = threadIdx.x; idx < K * nfc; idx += blockDim.x) {
        const int z = by_nfc.div(idx), fl = idx - z * nfc;
        const float4 v = line[(size_t)fl * M + (z >> 1)];
        dst[(size_t)z * nf + fl] = (z & 1) ? dfl{v.z, v.w} : dfl{v.x, v.y};
    }
}

// The k-space product of k_far_contract in double-float: derivatives and
// pair coefficients as double-float pairs, spectra as double-float complex;
// the scale 1/K^3 is a double-float pair (for K a power of two one float,
// exact on both halves).
__global__ void __launch_bounds__(256) k_far_contract_df(long long nq, int nout, const int* __restrict__ seg,
                                                         const FarPair* __restrict__ pairs,
                                                         const float2* __restrict__ pcoef,
                                                         const dfl* __restrict__ Dr, const float4* __restrict__ Mh,
                                                         float4* __restrict__ Th, float2 scale, bool pow2)
{
    const long long total = nq * nout;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(e / nq);
        const long long q = e - (long long)n * nq;
        dfl re = {0.0f, 0.0f}, im = {0.0f, 0.0f};
        const int e1 = seg[n + 1];
        for (int i = seg[n]; i < e1; ++i) {
            const FarPair pr = pairs[i];
            const float2 c = pcoef[i];
            const dfl cd = df_mul(dfl{c.x, c.y}, Dr[(size_t)(pr.j & 0x7fffffff) * nq + q]);
            const float4 m = Mh[(size_t)pr.k * nq + q];
            // odd |j|: i cd m = (-cd m.im, cd m.re)
            const bool odd = pr.j < 0;
            const dfl mr = odd ? dfl{m.z, m.w} : dfl{m.x, m.y}, mi = odd ? dfl{m.x, m.y} : dfl{m.z, m.w};
            re = df_fma(odd ? df_neg(cd) : cd, mr, re);
            im = df_fma(cd, mi, im);
        }
        if (pow2) {  // 1/K^3 is a power of two: exact on each half
            Th[e] = make_float4(re.h * scale.x, re.l * scale.x, im.h * scale.x, im.l * scale.x);
        } else {
            const dfl sc = {scale.x, scale.y};
            const dfl r = df_mul(re, sc), i = df_mul(im, sc);
            Th[e] = make_float4(r.h, r.l, i.h, i.l);
        }
    }
}

// FP64 -> double-float pairs, elementwise.
__global__ void k_to_df(const double* __restrict__ src, long long n, dfl* __restrict__ dst)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = df_from(src[i]);
}

// Cell multipoles in cell units, double-float, folded onto the reduced basis
// in the same kernel.  One block per cell and one thread per complete term:
// kMpChunk particles at a time the block builds their powers x^e, y^e, z^e
// (one thread per particle and axis) and the products x^a y^b (one per
// particle and (a, b) pair) in shared memory, and each term thread adds
// (x^a y^b) z^c to two double-float partial sums (updates without the
// renormalisation, df_fma_nr; the partial sums are added with df_add, which
// renormalises).  The cell's complete
// multipoles then go through the fold of k_far_reduce, Mr^r = sum_k
// f_{r,k} M^k, with its coefficients as double-float pairs, and are written
// as FP64 (Mr) or as double-float pairs (Mrd, for the double-float
// transforms), with the cell's (0,0,2) term for its sum over cells.  (The
// error-free transformations stay on scalar FP32 instructions: in probes the
// packed .f32x2 form of the same sequence did not always keep the product's
// rounding error, depending on the surrounding code.)
#ifndef NF_MP_CHUNK
#define NF_MP_CHUNK 32
#endif
constexpr int kMpChunk = NF_MP_CHUNK;
template <int P>
__global__ void k_multipoles_red_df(const int* __restrict__ off, const float4* __restrict__ rel, int C,
                                    const int* __restrict__ rseg, const int* __restrict__ rk,
                                    const double* __restrict__ rcoef, double* __restrict__ Mr,
                                    dfl* __restrict__ Mrd, double* __restrict__ m002)
{
    constexpr int P1 = P + 1, NAB = P1 * (P + 2) / 2, NT = far_terms(P), NR = P1 * P1;
    extern __shared__ dfl smem_mp[];
    const int nnz = rseg[NR];
    dfl* pw = smem_mp;                                  // powers [3][kMpChunk][P1]
    dfl* XY = pw + 3 * kMpChunk * P1;                   // products [kMpChunk][NAB]
    dfl* Ms = XY + kMpChunk * NAB;                      // the cell's complete multipoles [NT]
    dfl* cf = Ms + NT;                                  // fold coefficients [nnz]
    int2* abt = reinterpret_cast<int2*>(cf + nnz);      // (a, b) of each product [NAB]
    int* ck = reinterpret_cast<int*>(abt + NAB);        // complete term of each coefficient [nnz]
    int* sg = ck + nnz;                                 // segment of each reduced term [NR + 1]
    for (int i = threadIdx.x; i < nnz; i += blockDim.x) {
        cf[i] = df_from(rcoef[i]);
        ck[i] = rk[i];
    }
    for (int i = threadIdx.x; i <= NR; i += blockDim.x) sg[i] = rseg[i];
    for (int k = threadIdx.x; k < NAB; k += blockDim.x) {
        int aa = 0, kk = k;
        while (kk > P - aa) {
            kk -= P - aa + 1;
            ++aa;
        }
        abt[k] = make_int2(aa, kk);
    }
    int a = 0, b = 0, c = 0;
    const int t = threadIdx.x;
    if (t < NT) decode_term(t, P, a, b, c);
    const int ab = a * P1 - a * (a - 1) / 2 + b;
    const dfl* Z = pw + 2 * kMpChunk * P1;
    for (int cell = blockIdx.x; cell < C; cell += gridDim.x) {
        const int s0 = off[cell], s1 = off[cell + 1];
        // two independent partial sums: a double-float update is a chain of
        // dependent FP32 operations
        dfl acc0 = {0.0f, 0.0f}, acc1 = {0.0f, 0.0f};
        for (int q0 = s0; q0 < s1; q0 += kMpChunk) {
            const int nq = min(kMpChunk, s1 - q0);
            __syncthreads();  // the previous chunk (or the tables) are in place and read
            for (int i = threadIdx.x; i < 3 * nq; i += blockDim.x) {
                const int q = i / 3, d = i - 3 * q;
                const float4 r4 = rel[q0 + q];
                const float x = d == 0 ? r4.x : (d == 1 ? r4.y : r4.z);
                dfl* row = pw + (d * kMpChunk + q) * P1;
                dfl v = {x, 0.0f};
                row[0] = dfl{1.0f, 0.0f};
                if (P >= 1) row[1] = v;
#pragma unroll
                for (int e = 2; e <= P; ++e) {
                    v = df_mul_f(v, x);
                    row[e] = v;
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nq * NAB; i += blockDim.x) {
                const int q = i / NAB, k = i - q * NAB;
                const int2 ab2 = abt[k];
                XY[q * NAB + k] = df_mul(pw[q * P1 + ab2.x], pw[(kMpChunk + q) * P1 + ab2.y]);
            }
            __syncthreads();
            if (t < NT) {
                int q = 0;
                for (; q + 2 <= nq; q += 2) {
                    acc0 = df_fma_nr(XY[q * NAB + ab], Z[q * P1 + c], acc0);
                    acc1 = df_fma_nr(XY[(q + 1) * NAB + ab], Z[(q + 1) * P1 + c], acc1);
                }
                if (q < nq) acc0 = df_fma_nr(XY[q * NAB + ab], Z[q * P1 + c], acc0);
            }
        }
        if (t < NT) Ms[t] = df_add(acc0, acc1);
        __syncthreads();
        for (int r = threadIdx.x; r < NR; r += blockDim.x) {
            dfl m = {0.0f, 0.0f};
            for (int i = sg[r]; i < sg[r + 1]; ++i) m = df_fma(cf[i], Ms[ck[i]], m);
            if (Mrd)
                Mrd[(size_t)cell * NR + r] = m;  // the double-float transforms take the pairs as they are
            else
                Mr[(size_t)cell * NR + r] = (double)m.h + (double)m.l;
        }
        if (P >= 2 && t == 2) m002[cell] = (double)Ms[2].h + (double)Ms[2].l;  // term 2 is (0,0,2)
        __syncthreads();  // Ms is rewritten for the next cell
    }
}

// The Taylor evaluation of k_taylor_forces in double-float: cell units, the
// particle's stored FP32 offsets as the float multipliers of the Horner steps.
// Each thread evaluates two particles at once (binned slots i and i + half):
// a double-float Horner step is a chain of dependent FP32 operations, and two
// independent chains keep the FP32 pipe busy.  The steps skip the
// renormalisation (df_fma_f_nr, 11 instructions); the sums are converted to
// FP64 as hi + lo at the end.
__device__ __forceinline__ void store_far(int orig, double ax, double ay, double az, double* __restrict__ acc_far,
                                          float* __restrict__ acc_add)
{
    if (acc_far) {
        acc_far[3 * (size_t)orig] = ax;
        acc_far[3 * (size_t)orig + 1] = ay;
        acc_far[3 * (size_t)orig + 2] = az;
    }
    if (acc_add) {
        acc_add[3 * (size_t)orig] += (float)ax;
        acc_add[3 * (size_t)orig + 1] += (float)ay;
        acc_add[3 * (size_t)orig + 2] += (float)az;
    }
}

// The double-float Taylor evaluation's three Horner loops fully unrolled
// (compile-time term offsets: no index arithmetic in the loop body), or not.
#ifndef NF_TAYLOR_UNROLL
#define NF_TAYLOR_UNROLL 1
#endif
#if NF_TAYLOR_UNROLL
#define NF_TAYLOR_PRAGMA _Pragma("unroll")
#else
#define NF_TAYLOR_PRAGMA _Pragma("unroll 1")
#endif

template <int P>
__global__ void __launch_bounds__(128) k_taylor_forces_df(const int* __restrict__ cell, const float4* __restrict__ rel,
                                                         const dfl* __restrict__ T, int N, int C, double scale,
                                                         double* __restrict__ acc_far, float* __restrict__ acc_add)
{
    constexpr int NT = (P + 3) * (P + 2) * (P + 1) / 6;
    const dfl zero = {0.0f, 0.0f};
    const int half = (N + 1) / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < half; i += gridDim.x * blockDim.x) {
        const int j = i + half;                 // the second particle (may be past the end)
        const bool two = j < N;
        const int jj = two ? j : i;             // evaluate something valid, store only if two
        // the binning's sorted cell ids give each slot's cell (no search of the offsets)
        const dfl* __restrict__ T0 = T + (size_t)cell[i] * NT;
        const dfl* __restrict__ T1 = T + (size_t)cell[jj] * NT;
        const float4 r0 = rel[i], r1 = rel[jj];
        dfl F0 = zero, Fx0 = zero, Fy0 = zero, Fz0 = zero;
        dfl F1 = zero, Fx1 = zero, Fy1 = zero, Fz1 = zero;
NF_TAYLOR_PRAGMA
        for (int a = P; a >= 0; --a) {
            const int base_a = NT - (P - a + 3) * (P - a + 2) * (P - a + 1) / 6;
            dfl U0 = zero, Uy0 = zero, Uz0 = zero, U1 = zero, Uy1 = zero, Uz1 = zero;
NF_TAYLOR_PRAGMA
            for (int b = P - a; b >= 0; --b) {
                const int base = base_a + b * (P - a + 1) - b * (b - 1) / 2;
                dfl S0 = zero, Sz0 = zero, S1 = zero, Sz1 = zero;
NF_TAYLOR_PRAGMA
                for (int c = P - a - b; c >= 0; --c) {
                    const float2 t0 = __ldg(reinterpret_cast<const float2*>(T0 + base + c));
                    const float2 t1 = __ldg(reinterpret_cast<const float2*>(T1 + base + c));
                    Sz0 = df_fma_f_nr(Sz0, r0.z, S0);
                    Sz1 = df_fma_f_nr(Sz1, r1.z, S1);
                    S0 = df_fma_f_nr(S0, r0.z, dfl{t0.x, t0.y});
                    S1 = df_fma_f_nr(S1, r1.z, dfl{t1.x, t1.y});
                }
                Uy0 = df_fma_f_nr(Uy0, r0.y, U0);
                Uy1 = df_fma_f_nr(Uy1, r1.y, U1);
                U0 = df_fma_f_nr(U0, r0.y, S0);
                U1 = df_fma_f_nr(U1, r1.y, S1);
                Uz0 = df_fma_f_nr(Uz0, r0.y, Sz0);
                Uz1 = df_fma_f_nr(Uz1, r1.y, Sz1);
            }
            Fx0 = df_fma_f_nr(Fx0, r0.x, F0);
            Fx1 = df_fma_f_nr(Fx1, r1.x, F1);
            F0 = df_fma_f_nr(F0, r0.x, U0);
            F1 = df_fma_f_nr(F1, r1.x, U1);
            Fy0 = df_fma_f_nr(Fy0, r0.x, Uy0);
            Fy1 = df_fma_f_nr(Fy1, r1.x, Uy1);
            Fz0 = df_fma_f_nr(Fz0, r0.x, Uz0);
            Fz1 = df_fma_f_nr(Fz1, r1.x, Uz1);
        }
        store_far(__float_as_int(r0.w), scale * ((double)Fx0.h + (double)Fx0.l),
                  scale * ((double)Fy0.h + (double)Fy0.l), scale * ((double)Fz0.h + (double)Fz0.l), acc_far,
                  acc_add);
        if (two)
            store_far(__float_as_int(r1.w), scale * ((double)Fx1.h + (double)Fx1.l),
                      scale * ((double)Fy1.h + (double)Fy1.l), scale * ((double)Fz1.h + (double)Fz1.l), acc_far,
                      acc_add);
    }
}

// Taylors in box units from cell units: T^n = T'^n / w^{|n|}, [C][nt].
__global__ void k_unscale_taylors(const double* __restrict__ Tc, long long total, int nt, int p, double inv_w,
                                  double* __restrict__ T)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int a, b, c;
        decode_term((int)(e % nt), p, a, b, c);
        double f = 1.0;
        for (int i = 0; i < a + b + c; ++i) f *= inv_w;
        T[e] = Tc[e] * f;
    }
}

// Fold of the complete multipoles onto the reduced ones: Mr[c][r] =
// sum_{entries of r} coef * M[c][k]; one thread per (cell, reduced term).
__global__ void k_far_reduce(const double* __restrict__ M, int C, int nt, int nr, const int* __restrict__ seg,
                             const int* __restrict__ kidx, const double* __restrict__ coef, double* __restrict__ Mr)
{
    const long long total = (long long)C * nr;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long c = e / nr;
        const int r = (int)(e - c * nr);
        const double* m = M + c * nt;
        double acc = 0.0;
        for (int i = seg[r]; i < seg[r + 1]; ++i) acc = fma(coef[i], m[kidx[i]], acc);
        Mr[e] = acc;
    }
}

// Partial sums over cells of M[c][term], one per block (gridDim.x of them),
// each in a fixed order; the rebuild adds the partials in order.
constexpr int kSumBlocks = 64;
__global__ void k_far_sum_term(const double* __restrict__ M, int C, int nt, int term, double* __restrict__ partial)
{
    __shared__ double part[256];
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x)
        acc += M[(size_t)c * nt + term];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = part[0];
}

// Complete Taylors of every cell from the reduced ones: one warp per cell,
// the rebuild program in shared memory and the cell's Taylors staged in a
// per-warp shared buffer.  The warp reads a cell's reduced Taylors in one
// coalesced pass (fetching the next cell's into registers while it rebuilds
// the current one) and drops each into its place in the complete basis: the
// terms with z index 0 and 1 are the reduced ones.  The rest of the program
// is ordered by the z index of its destination; ops of one z level are
// independent (their sources have z - 2), so the lanes share a level and
// sync between levels.  lap is the Laplacian of the series (4 pi N w^2 / V in
// cell units); t0_per_s002 times the sum of the partials is the constant of
// T^0.  F64 runs the recursion in FP64 and writes T; DF splits the reduced
// Taylors into double-float pairs once and runs the recursion on the FP32
// pipe, writing Tdf: the forces of the double-float kernels do not depend on
// whether T is asked for too.  DIN: the reduced Taylors arrive as
// double-float pairs (from the double-float transforms) instead of FP64.
constexpr int kRebuildWarps = 8;
constexpr int kRebuildFetch = (kMaxFarOrder + 1) * (kMaxFarOrder + 1) / 32 + 1;  // reduced terms per lane
template <bool F64, bool DF, bool DIN>
__global__ void k_far_rebuild(const void* __restrict__ Trv, int C, int p, int nt, int nr, const int4* __restrict__ ops,
                              const double2* __restrict__ opf, int t002, double lap, double t0_per_s002,
                              const double* __restrict__ partial, double* __restrict__ T, dfl* __restrict__ Tdf)
{
    extern __shared__ int4 smem_rb[];
    int4* prog = smem_rb;                                     // [nt] ops
    double2* fs = reinterpret_cast<double2*>(prog + nt);      // [nt] factors
    float4* fd = reinterpret_cast<float4*>(fs + nt);          // [nt] factors as double-float pairs
    int* level = reinterpret_cast<int*>(fd + nt);             // [16] level starts
    int* rmap = level + 16;                                   // [nr] place of each reduced term
    double* stage = reinterpret_cast<double*>(rmap + ((nr + 3) & ~3));  // per warp: [nt] FP64, [nt] pairs
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        const int4 op = ops[i];
        prog[i] = op;
        if (op.y >= 0) rmap[op.y] = op.x;
        const double2 f = opf[i];
        fs[i] = f;
        const dfl x = df_from(f.x), y = df_from(f.y);
        fd[i] = make_float4(x.h, x.l, y.h, y.l);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int i = 0;
        for (int c = 0; c <= p; ++c) {
            level[c] = i;
            while (i < nt) {
                int a, b, cz;
                decode_term(prog[i].x, p, a, b, cz);
                if (cz != c) break;
                ++i;
            }
        }
        level[p + 1] = nt;
    }
    __syncthreads();
    double t0 = 0.0;
    if (t002 >= 0 && partial)
        for (int q = 0; q < kSumBlocks; ++q) t0 += partial[q];
    t0 *= t0_per_s002;
    const dfl t0d = df_from(t0), lapd = df_from(0.5 * lap);
    const int lane = threadIdx.x & 31;
    double* t = stage + (size_t)(threadIdx.x >> 5) * ((F64 ? 1 : 0) + (DF ? 1 : 0)) * nt;
    dfl* td = reinterpret_cast<dfl*>(t + (F64 ? nt : 0));
    int rdst[kRebuildFetch];
#pragma unroll
    for (int k = 0; k < kRebuildFetch; ++k) rdst[k] = lane + 32 * k < nr ? rmap[lane + 32 * k] : -1;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    // the reduced Taylors as raw 8-byte words: an FP64 value, or a double-float pair (DIN)
    const unsigned long long* __restrict__ Tr = static_cast<const unsigned long long*>(Trv);
    unsigned long long nx[kRebuildFetch];
    int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
#pragma unroll
    for (int k = 0; k < kRebuildFetch; ++k) {
        const int i = lane + 32 * k;
        nx[k] = (c < C && i < nr) ? Tr[(size_t)c * nr + i] : 0ull;
    }
    for (; c < C; c += warps) {
#pragma unroll
        for (int k = 0; k < kRebuildFetch; ++k) {
            const int d = rdst[k];
            if (d >= 0) {
                const dfl vd = DIN ? dfl{__uint_as_float((unsigned)nx[k]), __uint_as_float((unsigned)(nx[k] >> 32))}
                                   : df_from(__longlong_as_double((long long)nx[k]));
                const double v = DIN ? (double)vd.h + (double)vd.l : __longlong_as_double((long long)nx[k]);
                if (F64) t[d] = d == 0 ? v + t0 : v;
                if (DF) td[d] = d == 0 ? df_add(vd, t0d) : vd;
            }
        }
        __syncwarp();
        const int cn = c + warps;
#pragma unroll
        for (int k = 0; k < kRebuildFetch; ++k) {
            const int i = lane + 32 * k;
            nx[k] = (cn < C && i < nr) ? Tr[(size_t)cn * nr + i] : 0ull;
        }
        for (int L = 2; L <= p; ++L) {
            for (int i = level[L] + lane; i < level[L + 1]; i += 32) {
                const int4 op = prog[i];
                if (F64) {
                    double v = -fs[i].x * t[op.z] - fs[i].y * t[op.w];
                    if (op.x == t002) v += 0.5 * lap;  // m = 0: (2)(1) T^{002} = lap - ...
                    t[op.x] = v;
                }
                if (DF) {
                    const float4 f = fd[i];
                    dfl v = df_fma(dfl{f.x, f.y}, td[op.z], df_mul(dfl{f.z, f.w}, td[op.w]));
                    v = dfl{-v.h, -v.l};
                    if (op.x == t002) v = df_add(v, lapd);
                    td[op.x] = v;
                }
            }
            __syncwarp();
        }
        if (F64)
            for (int i = lane; i < nt; i += 32) T[(size_t)c * nt + i] = t[i];
        if (DF)
            for (int i = lane; i < nt; i += 32) Tdf[(size_t)c * nt + i] = td[i];
        __syncwarp();  // the buffers are reused by the next cell
    }
}

__global__ void k_deriv_header(DerivHeader h, DerivHeader* dst)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *dst = h;
}

int device_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}


}  // namespace

int far_terms_host(int p) { return far_terms(p); }

// Reduced basis (Sec. "Far-field Computation": the paper converts the
// multipoles to a reduced basis of (p+1)^2 values before the FFTs).  Away from
// the lattice points every trace of the derivatives vanishes except the
// second-order one, which is the background's 4 pi / V:
//     D^{i+2ex} + D^{i+2ey} + D^{i+2ez} = (4 pi / V) [i = 0],
// so D^{n+k} with k_z >= 2 equals -D^{n+k-2ez+2ex} - D^{n+k-2ez+2ey} (plus
// 4 pi/V when n + k = 2ez, a constant potential in every cell).  Applied
// repeatedly this folds every multipole onto the terms with k_z <= 1 (same
// order |k|, so the truncation |n| + |k| <= p is kept): the convolution and
// its FFTs run on (p+1)^2 fields.  The Taylors are computed for the reduced
// n the same way and the rest rebuilt per cell from the Laplacian of the
// truncated series, which is exactly 4 pi N / V (the same identity summed
// over the sources):  (m_x+2)(m_x+1) T^{m+2ex} + (m_y+2)(m_y+1) T^{m+2ey}
// + (m_z+2)(m_z+1) T^{m+2ez} = (4 pi N / V) [m = 0].  The constant the fold
// drops from T^0 is added back from the sum of the (0,0,2) multipoles.
FarTables far_tables(int p, double w)
{
    FarTables tb;
    const int nt = far_terms(p);
    std::vector<int> ta(nt), tbv(nt), tc(nt), rindex(nt, -1);
    {
        int t = 0;
        for (int a = 0; a <= p; ++a)
            for (int b = 0; b <= p - a; ++b)
                for (int c = 0; c <= p - a - b; ++c, ++t) {
                    ta[t] = a;
                    tbv[t] = b;
                    tc[t] = c;
                    if (c <= 1) rindex[t] = tb.nr++;
                }
    }
    double fac[2 * kMaxFarOrder + 2];
    fac[0] = 1.0;
    for (int i = 1; i <= 2 * kMaxFarOrder + 1; ++i) fac[i] = fac[i - 1] * i;
    // E(k): the reduced terms D^{n+k} folds onto, with integer coefficients
    std::vector<std::map<int, double>> E(nt);
    for (int c = 0; c <= p; ++c)  // by k_z, so the folded terms are known first
        for (int t = 0; t < nt; ++t) {
            if (tc[t] != c) continue;
            if (c <= 1) {
                E[t][rindex[t]] = 1.0;
                continue;
            }
            const int s1 = encode_term(ta[t] + 2, tbv[t], c - 2, p), s2 = encode_term(ta[t], tbv[t] + 2, c - 2, p);
            for (const auto& kv : E[s1]) E[t][kv.first] -= kv.second;
            for (const auto& kv : E[s2]) E[t][kv.first] -= kv.second;
        }
    // the fold, grouped by reduced term: Mr^r = sum_k (-1)^{|k|} / k! E(k)_r M^k
    std::vector<std::vector<std::pair<int, double>>> by_r(tb.nr);
    for (int t = 0; t < nt; ++t) {
        const double wk = (((ta[t] + tbv[t] + tc[t]) & 1) ? -1.0 : 1.0) / (fac[ta[t]] * fac[tbv[t]] * fac[tc[t]]);
        for (const auto& kv : E[t])
            if (kv.second != 0.0) by_r[kv.first].push_back({t, wk * kv.second});
    }
    tb.red_seg.push_back(0);
    for (int r = 0; r < tb.nr; ++r) {
        for (const auto& e : by_r[r]) {
            tb.red_k.push_back(e.first);
            tb.red_coef.push_back(e.second);
        }
        tb.red_seg.push_back((int)tb.red_k.size());
    }
    // reduced pairs: T^n = w^{|n|+|k|} / n! D^{n+k} Mr^k, n and k reduced, |n| + |k| <= p
    std::vector<double> wp(2 * kMaxFarOrder + 1, 1.0);
    for (int i = 1; i <= p; ++i) wp[i] = wp[i - 1] * w;
    tb.pair_seg.push_back(0);
    for (int n = 0; n < nt; ++n) {
        if (rindex[n] < 0) continue;
        for (int k = 0; k < nt; ++k) {
            if (rindex[k] < 0) continue;
            const int order = ta[n] + tbv[n] + tc[n] + ta[k] + tbv[k] + tc[k];
            if (order > p) continue;
            FarPair pr;
            pr.k = rindex[k];
            pr.j = encode_term(ta[n] + ta[k], tbv[n] + tbv[k], tc[n] + tc[k], p);
            if (order & 1) pr.j |= (int)0x80000000u;
            pr.coef = wp[order] / (fac[ta[n]] * fac[tbv[n]] * fac[tc[n]]);
            tb.pairs.push_back(pr);
            const float ch = (float)pr.coef;
            tb.pair_cdf.push_back(make_float2(ch, (float)(pr.coef - (double)ch)));
        }
        tb.pair_seg.push_back((int)tb.pairs.size());
    }
    // rebuild program, by z index: copies of the reduced Taylors, then the recursion
    for (int c = 0; c <= p; ++c)
        for (int t = 0; t < nt; ++t) {
            if (tc[t] != c) continue;
            if (c <= 1) {
                tb.ops.push_back(make_int4(t, rindex[t], 0, 0));
                tb.opf.push_back(make_double2(0.0, 0.0));
                continue;
            }
            const int a = ta[t], b = tbv[t];
            const double inv = 1.0 / (double)(c * (c - 1));
            tb.ops.push_back(make_int4(t, -1, encode_term(a + 2, b, c - 2, p), encode_term(a, b + 2, c - 2, p)));
            tb.opf.push_back(make_double2((a + 2) * (a + 1) * inv, (b + 2) * (b + 1) * inv));
        }
    tb.t002 = p >= 2 ? encode_term(0, 0, 2, p) : -1;
    return tb;
}

// ---- mixed-radix transforms for any K ---------------------------------------
// The same 3-D real transforms as above (layouts of the power-of-two kernels:
// real side cell-major [x][y][z][field], spectrum [field][x][y][kz], kz <=
// K/2; forward e^{-i...}, the inverse unnormalised) for any K, in IEEE FP64
// (the derivatives tensor, and the FP64 mode) or in double-float (K not a
// power of two).  Each 1-D transform runs on lines held in shared memory as a
// self-sorting Stockham sequence of radix-R steps over the factors of K
// (fours first, then 2, 3, 5, 7, then any larger prime): with Ns the product
// of the radices already done, step j (j < K/R) reads a[j + r K/R] times
// W_K^{r k K/(Ns R)} (k = j mod Ns) for r < R, forms their R-point DFT by
// definition (roots W_K^{(q m mod R) K/R}), and writes it to
// y[(j - k) R + k + m Ns]; natural order in and out, two buffers in turn.
// The real z lines are transformed as complex lines with zero imaginary
// parts; the inverse z pass rebuilds the whole Hermitian line from kz <= K/2
// (dropping the imaginary parts at kz = 0 and K/2, as a complex-to-real
// transform does) and keeps the real parts.
namespace {

struct ArF64 {
    typedef double real_t;
    typedef double2 spec_t;
    struct cx {
        double re, im;
    };
    static __device__ __forceinline__ cx ld(spec_t v) { return {v.x, v.y}; }
    static __device__ __forceinline__ spec_t st(cx v) { return make_double2(v.re, v.im); }
    static __device__ __forceinline__ cx from_real(real_t v) { return {v, 0.0}; }
    static __device__ __forceinline__ real_t real(cx v) { return v.re; }
    static __device__ __forceinline__ cx conj(cx v) { return {v.re, -v.im}; }
    static __device__ __forceinline__ cx no_im(cx v) { return {v.re, 0.0}; }
    static __device__ __forceinline__ cx add(cx a, cx b) { return {a.re + b.re, a.im + b.im}; }
    static __device__ __forceinline__ cx mul(cx w, cx x)
    {
        return {fma(w.re, x.re, -w.im * x.im), fma(w.re, x.im, w.im * x.re)};
    }
};

struct ArDF {
    typedef dfl real_t;
    typedef float4 spec_t;
    typedef cdf cx;
    static __device__ __forceinline__ cx ld(spec_t v) { return cdf_ld(v); }
    static __device__ __forceinline__ spec_t st(cx v) { return cdf_st(v); }
    static __device__ __forceinline__ cx from_real(real_t v) { return {v, dfl{0.0f, 0.0f}}; }
    static __device__ __forceinline__ real_t real(cx v) { return v.re; }
    static __device__ __forceinline__ cx conj(cx v) { return {v.re, df_neg(v.im)}; }
    static __device__ __forceinline__ cx no_im(cx v) { return {v.re, dfl{0.0f, 0.0f}}; }
    static __device__ __forceinline__ cx add(cx a, cx b) { return cdf_add(a, b); }
    static __device__ __forceinline__ cx mul(cx w, cx x) { return cdf_mul(w, x); }
};

constexpr int kGPoints = 1024;  // complex points per buffer of one block

__host__ __device__ inline int gfft_lines_per_block(int K) { return K >= kGPoints ? 1 : kGPoints / K; }

template <class A, bool INV>
__device__ __forceinline__ typename A::cx gtw(const typename A::cx* tw, int j)
{
    return INV ? A::conj(tw[j]) : tw[j];
}

// One radix-R step for the point j of a line (R known at compile time).
template <class A, bool INV, int R>
__device__ __forceinline__ void gfft_step(const typename A::cx* a, typename A::cx* y, const typename A::cx* tw, int K,
                                          int KR, int Ns, int j)
{
    typedef typename A::cx cx;
    const int k = j % Ns, step = KR / Ns;  // K / (Ns R)
    cx v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const cx x = a[j + r * KR];
        v[r] = r ? A::mul(gtw<A, INV>(tw, r * k * step), x) : x;
    }
    const int o = (j - k) * R + k;
#pragma unroll
    for (int m = 0; m < R; ++m) {
        cx acc = v[0];
#pragma unroll
        for (int q = 1; q < R; ++q) acc = A::add(acc, A::mul(gtw<A, INV>(tw, ((q * m) % R) * KR), v[q]));
        y[o + m * Ns] = acc;
    }
}

// The same for a radix known only at run time (a prime factor above 7).
template <class A, bool INV>
__device__ void gfft_step_any(const typename A::cx* a, typename A::cx* y, const typename A::cx* tw, int K, int R,
                              int KR, int Ns, int j)
{
    typedef typename A::cx cx;
    const int k = j % Ns, step = KR / Ns;
    const int o = (j - k) * R + k;
    for (int m = 0; m < R; ++m) {
        cx acc = a[j];
        for (int q = 1; q < R; ++q) {
            const cx x = A::mul(gtw<A, INV>(tw, q * k * step), a[j + q * KR]);
            acc = A::add(acc, A::mul(gtw<A, INV>(tw, ((q * m) % R) * KR), x));
        }
        y[o + m * Ns] = acc;
    }
}

// Transforms nl lines of K points in b0 (natural order); returns the buffer
// that holds the result (b0 or b1).
template <class A, bool INV>
__device__ typename A::cx* gfft_stages(typename A::cx* b0, typename A::cx* b1, int nl, int K, const Radices& rd,
                                       const typename A::cx* tw)
{
    typedef typename A::cx cx;
    cx* src = b0;
    cx* dst = b1;
    int Ns = 1;
    for (int st = 0; st < rd.n; ++st) {
        const int R = rd.r[st], KR = K / R;
        for (int idx = threadIdx.x; idx < nl * KR; idx += blockDim.x) {
            const int l = idx / KR, j = idx - l * KR;
            const cx* a = src + (size_t)l * K;
            cx* y = dst + (size_t)l * K;
            switch (R) {
                case 2: gfft_step<A, INV, 2>(a, y, tw, K, KR, Ns, j); break;
                case 3: gfft_step<A, INV, 3>(a, y, tw, K, KR, Ns, j); break;
                case 4: gfft_step<A, INV, 4>(a, y, tw, K, KR, Ns, j); break;
                case 5: gfft_step<A, INV, 5>(a, y, tw, K, KR, Ns, j); break;
                case 7: gfft_step<A, INV, 7>(a, y, tw, K, KR, Ns, j); break;
                default: gfft_step_any<A, INV>(a, y, tw, K, R, KR, Ns, j); break;
            }
        }
        __syncthreads();
        cx* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// Shared memory of the generic kernels: the K twiddles, then two buffers of
// (lines per block) x K points.
template <class A>
__host__ __device__ size_t gfft_smem(int K)
{
    return sizeof(typename A::cx) * ((size_t)K + 2ull * gfft_lines_per_block(K) * K);
}

// Forward z pass: real fields R [x][y][z][nf] -> spectrum S [nf][x][y][kz].
template <class A>
__global__ void __launch_bounds__(kFftThreads) k_gfft_z_fwd(const typename A::real_t* __restrict__ Rf, int K, int nf,
                                                            int nchunk, Radices rd,
                                                            const typename A::spec_t* __restrict__ twg,
                                                            typename A::spec_t* __restrict__ S)
{
    typedef typename A::cx cx;
    extern __shared__ __align__(16) unsigned char gsm[];
    cx* tw = reinterpret_cast<cx*>(gsm);
    const int FB = gfft_lines_per_block(K), H = K / 2 + 1;
    cx* b0 = tw + K;
    cx* b1 = b0 + (size_t)FB * K;
    const int chunk = blockIdx.x % nchunk;
    const long long xy = blockIdx.x / nchunk;
    const int f0 = chunk * FB, nfc = min(FB, nf - f0);
    for (int j = threadIdx.x; j < K; j += blockDim.x) tw[j] = A::ld(twg[j]);
    const typename A::real_t* src = Rf + (size_t)xy * K * nf + f0;
    for (int idx = threadIdx.x; idx < K * nfc; idx += blockDim.x) {
        const int z = idx / nfc, fl = idx - z * nfc;
        b0[(size_t)fl * K + z] = A::from_real(src[(size_t)z * nf + fl]);
    }
    __syncthreads();
    const cx* out = gfft_stages<A, false>(b0, b1, nfc, K, rd, tw);
    const size_t fstride = (size_t)K * K * H;
    for (int idx = threadIdx.x; idx < nfc * H; idx += blockDim.x) {
        const int fl = idx / H, k = idx - fl * H;
        S[(size_t)(f0 + fl) * fstride + (size_t)xy * H + k] = A::st(out[(size_t)fl * K + k]);
    }
}

// Complex passes along y or x, in place on S (as k_fft_lines).
template <class A, bool INV>
__global__ void __launch_bounds__(kFftThreads) k_gfft_lines(typename A::spec_t* __restrict__ S, int K, int nA,
                                                            long long astride, long long pstride, int nchunk,
                                                            Radices rd, const typename A::spec_t* __restrict__ twg)
{
    typedef typename A::cx cx;
    extern __shared__ __align__(16) unsigned char gsm[];
    cx* tw = reinterpret_cast<cx*>(gsm);
    const int W = gfft_lines_per_block(K), H = K / 2 + 1;
    cx* b0 = tw + K;
    cx* b1 = b0 + (size_t)W * K;
    const int chunk = blockIdx.x % nchunk;
    const long long fa = blockIdx.x / nchunk;
    const long long f = fa / nA, a = fa - f * nA;
    const int k0 = chunk * W, wc = min(W, H - k0);
    for (int j = threadIdx.x; j < K; j += blockDim.x) tw[j] = A::ld(twg[j]);
    typename A::spec_t* base = S + f * (long long)K * K * H + a * astride + k0;
    for (int idx = threadIdx.x; idx < K * wc; idx += blockDim.x) {
        const int pt = idx / wc, w = idx - pt * wc;
        b0[(size_t)w * K + pt] = A::ld(base[pt * pstride + w]);
    }
    __syncthreads();
    const cx* out = gfft_stages<A, INV>(b0, b1, wc, K, rd, tw);
    for (int idx = threadIdx.x; idx < K * wc; idx += blockDim.x) {
        const int pt = idx / wc, w = idx - pt * wc;
        base[pt * pstride + w] = A::st(out[(size_t)w * K + pt]);
    }
}

// Inverse z pass: spectrum S (kz <= K/2) -> real fields R [x][y][z][nf].
template <class A>
__global__ void __launch_bounds__(kFftThreads) k_gfft_z_inv(const typename A::spec_t* __restrict__ S, int K, int nf,
                                                            int nchunk, Radices rd,
                                                            const typename A::spec_t* __restrict__ twg,
                                                            typename A::real_t* __restrict__ Rf)
{
    typedef typename A::cx cx;
    extern __shared__ __align__(16) unsigned char gsm[];
    cx* tw = reinterpret_cast<cx*>(gsm);
    const int FB = gfft_lines_per_block(K), H = K / 2 + 1;
    cx* b0 = tw + K;
    cx* b1 = b0 + (size_t)FB * K;
    const int chunk = blockIdx.x % nchunk;
    const long long xy = blockIdx.x / nchunk;
    const int f0 = chunk * FB, nfc = min(FB, nf - f0);
    for (int j = threadIdx.x; j < K; j += blockDim.x) tw[j] = A::ld(twg[j]);
    const size_t fstride = (size_t)K * K * H;
    for (int idx = threadIdx.x; idx < nfc * K; idx += blockDim.x) {
        const int fl = idx / K, k = idx - fl * K;
        const typename A::spec_t* row = S + (size_t)(f0 + fl) * fstride + (size_t)xy * H;
        cx v;
        if (k < H) {
            v = A::ld(row[k]);
            if (k == 0 || 2 * k == K) v = A::no_im(v);
        } else {
            v = A::conj(A::ld(row[K - k]));  // Hermitian symmetry of a real field
        }
        b0[(size_t)fl * K + k] = v;
    }
    __syncthreads();
    const cx* out = gfft_stages<A, true>(b0, b1, nfc, K, rd, tw);
    typename A::real_t* dst = Rf + (size_t)xy * K * nf + f0;
    for (int idx = threadIdx.x; idx < K * nfc; idx += blockDim.x) {
        const int z = idx / nfc, fl = idx - z * nfc;
        dst[(size_t)z * nf + fl] = A::real(out[(size_t)fl * K + z]);
    }
}

template <class A>
cudaError_t launch_gfft(int K, int nf, bool forward, const void* real_in, void* spec, void* real_out, const void* tw,
                        cudaStream_t s)
{
    typedef typename A::spec_t spec_t;
    typedef typename A::real_t real_t;
    const Radices rd = far_radices(K);
    const int H = K / 2 + 1, FB = gfft_lines_per_block(K);
    const size_t smem = gfft_smem<A>(K);
    const spec_t* twg = static_cast<const spec_t*>(tw);
    spec_t* S = static_cast<spec_t*>(spec);
    const int zchunks = (nf + FB - 1) / FB, lchunks = (H + FB - 1) / FB;
    const long long zblocks = (long long)K * K * zchunks, lblocks = (long long)nf * K * lchunks;
    const long long KH = (long long)K * H;
    cudaError_t e;
    if (forward) {
        e = ensure_smem((const void*)k_gfft_z_fwd<A>, (int)smem);
        if (e == cudaSuccess) e = ensure_smem((const void*)k_gfft_lines<A, false>, (int)smem);
        if (e != cudaSuccess) return e;
        k_gfft_z_fwd<A><<<(unsigned)zblocks, kFftThreads, smem, s>>>(static_cast<const real_t*>(real_in), K, nf,
                                                                      zchunks, rd, twg, S);
        k_gfft_lines<A, false><<<(unsigned)lblocks, kFftThreads, smem, s>>>(S, K, K, KH, H, lchunks, rd, twg);
        k_gfft_lines<A, false><<<(unsigned)lblocks, kFftThreads, smem, s>>>(S, K, K, H, KH, lchunks, rd, twg);
    } else {
        e = ensure_smem((const void*)k_gfft_z_inv<A>, (int)smem);
        if (e == cudaSuccess) e = ensure_smem((const void*)k_gfft_lines<A, true>, (int)smem);
        if (e != cudaSuccess) return e;
        k_gfft_lines<A, true><<<(unsigned)lblocks, kFftThreads, smem, s>>>(S, K, K, H, KH, lchunks, rd, twg);
        k_gfft_lines<A, true><<<(unsigned)lblocks, kFftThreads, smem, s>>>(S, K, K, KH, H, lchunks, rd, twg);
        k_gfft_z_inv<A><<<(unsigned)zblocks, kFftThreads, smem, s>>>(S, K, nf, zchunks, rd, twg,
                                                                      static_cast<real_t*>(real_out));
    }
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace

Radices far_radices(int K)
{
    Radices rd{};
    int n = K;
    auto push = [&](int r) { rd.r[rd.n++] = r; };
    while (n % 4 == 0) {
        push(4);
        n /= 4;
    }
    for (int r : {2, 3, 5, 7}) {
        while (n % r == 0) {
            push(r);
            n /= r;
        }
    }
    for (int r = 11; n > 1; r += 2) {
        while (n % r == 0) {
            push(r);
            n /= r;
        }
    }
    return rd;
}

std::vector<double2> far_twiddles64(int K)
{
    std::vector<double2> tw(K);
    for (int j = 0; j < K; ++j) {
        const double th = 2.0 * 3.14159265358979323846 * j / K;
        tw[j] = make_double2(std::cos(th), -std::sin(th));
    }
    return tw;
}

cudaError_t launch_far_fft64(int K, int nf, bool forward, const double* real_in, double2* spec, double* real_out,
                             const double2* tw, cudaStream_t s)
{
    return launch_gfft<ArF64>(K, nf, forward, real_in, spec, real_out, tw, s);
}


cudaError_t launch_deriv_real(int K, int R, int p, double box, double alpha, int nimg, double* D, cudaStream_t s)
{
    const int nt = far_terms(p);
    const size_t smem = deriv_real_smem(p);
    cudaError_t e = ensure_smem((const void*)k_deriv_real, (int)smem);
    if (e != cudaSuccess) return e;
    const int C = K * K * K;
    const int grid = C < device_sms() * 8 ? C : device_sms() * 8;
    k_deriv_real<<<grid, kDerivThreads, smem, s>>>(K, R, p, nt, box, alpha, nimg, D);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_deriv_recip(int K, int p, double box, double alpha, int hmax, const double2* Dh, double* Dr,
                               cudaStream_t s)
{
    const int nt = far_terms(p);
    const long long total = (long long)nt * K * K * (K / 2 + 1);
    long long blocks = (total + 255) / 256;
    const long long cap = (long long)device_sms() * 16;
    if (blocks > cap) blocks = cap;
    k_deriv_recip<<<(int)blocks, 256, 0, s>>>(K, p, nt, box, alpha, hmax, Dh, Dr);
    count_launches(1);
    return cudaGetLastError();
}

bool far_df_fft(int K) { return K >= 4 && K <= 256 && (K & (K - 1)) == 0; }

std::vector<float4> far_twiddles(int K)
{
    std::vector<float4> tw(K);
    for (int j = 0; j < K; ++j) {
        const double th = 2.0 * 3.14159265358979323846 * j / K;
        const double c = std::cos(th), sn = -std::sin(th);
        const float ch = (float)c, sh = (float)sn;
        tw[j] = make_float4(ch, (float)(c - (double)ch), sh, (float)(sn - (double)sh));
    }
    return tw;
}

cudaError_t launch_far_fft_df(int K, int nf, bool forward, const void* real_in, void* spec, void* real_out,
                              const void* tw, cudaStream_t s)
{
    if (!far_df_fft(K)) return launch_gfft<ArDF>(K, nf, forward, real_in, spec, real_out, tw, s);
    int logK = 0;
    while ((1 << logK) < K) ++logK;
    const int H = K / 2 + 1, FB = fft_lines_per_block(K), FBz = fft_z_lines_per_block(K);
    // the same points per block for both kinds of pass: FB lines of K or FBz lines of K/2
    const size_t smem = ((size_t)K / 2 + (size_t)FB * K) * sizeof(float4);
    const float4* twg = static_cast<const float4*>(tw);
    float4* S = static_cast<float4*>(spec);
    const int zchunks = (nf + FBz - 1) / FBz, lchunks = (H + FB - 1) / FB;
    const long long zblocks = (long long)K * K * zchunks, lblocks = (long long)nf * K * lchunks;
    const long long KH = (long long)K * H;
    cudaError_t e;
    if (forward) {
        e = ensure_smem((const void*)k_fft_z_fwd, (int)smem);
        if (e == cudaSuccess) e = ensure_smem((const void*)k_fft_lines<false>, (int)smem);
        if (e != cudaSuccess) return e;
        k_fft_z_fwd<<<(unsigned)zblocks, kFftThreads, smem, s>>>(static_cast<const dfl*>(real_in), K, logK, nf,
                                                                  zchunks, twg, S);
        // y lines: per (field, x), points H apart; x lines: per (field, y), points K H apart
        k_fft_lines<false><<<(unsigned)lblocks, kFftThreads, smem, s>>>(S, K, logK, K, KH, H, lchunks, twg);
        k_fft_lines<false><<<(unsigned)lblocks, kFftThreads, smem, s>>>(S, K, logK, K, H, KH, lchunks, twg);
    } else {
        e = ensure_smem((const void*)k_fft_z_inv, (int)smem);
        if (e == cudaSuccess) e = ensure_smem((const void*)k_fft_lines<true>, (int)smem);
        if (e != cudaSuccess) return e;
        k_fft_lines<true><<<(unsigned)lblocks, kFftThreads, smem, s>>>(S, K, logK, K, H, KH, lchunks, twg);
        k_fft_lines<true><<<(unsigned)lblocks, kFftThreads, smem, s>>>(S, K, logK, K, KH, H, lchunks, twg);
        k_fft_z_inv<<<(unsigned)zblocks, kFftThreads, smem, s>>>(S, K, logK, nf, zchunks, twg,
                                                                  static_cast<dfl*>(real_out));
    }
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_far_contract_df(int K, int nout, const int* seg, const FarPair* pairs, const void* pcoef,
                                   const void* Dr, const void* Mh, void* Th, cudaStream_t s)
{
    const long long nq = (long long)K * K * (K / 2 + 1);
    long long blocks = (nq * nout + 255) / 256;
    const long long cap = (long long)device_sms() * 64;
    if (blocks > cap) blocks = cap;
    // the unnormalised inverse transform's 1/K^3, as a double-float pair (one float when K = 2^n)
    const double sd = 1.0 / ((double)K * K * K);
    const float sh = (float)sd;
    const float2 scale = make_float2(sh, (float)(sd - (double)sh));
    const bool pow2 = (K & (K - 1)) == 0;
    k_far_contract_df<<<(int)blocks, 256, 0, s>>>(nq, nout, seg, pairs, static_cast<const float2*>(pcoef),
                                                  static_cast<const dfl*>(Dr), static_cast<const float4*>(Mh),
                                                  static_cast<float4*>(Th), scale, pow2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_to_df(const double* src, long long n, void* dst, cudaStream_t s)
{
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)device_sms() * 32;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) return cudaSuccess;
    k_to_df<<<(int)blocks, 256, 0, s>>>(src, n, static_cast<dfl*>(dst));
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_multipoles_red_df(const int* off, const float4* rel, int C, int p, const int* rseg,
                                     const int* rk, const double* rcoef, long long nnz, double* Mr, void* Mrd,
                                     double* m002, cudaStream_t s)
{
    const int nt = far_terms(p), nr = (p + 1) * (p + 1), nab = (p + 1) * (p + 2) / 2;
    const int threads = ((nt + 31) / 32) * 32;
    const size_t smem = ((size_t)3 * kMpChunk * (p + 1) + (size_t)kMpChunk * nab + nt + nnz) * sizeof(dfl) +
                        (size_t)nab * sizeof(int2) + ((size_t)nnz + nr + 1) * sizeof(int);
    const int grid = C < device_sms() * 32 ? C : device_sms() * 32;
    switch (p) {
#define NF_MP_RED_CASE(P)                                                                              \
    case P: {                                                                                          \
        cudaError_t e = ensure_smem((const void*)k_multipoles_red_df<P>, (int)smem);                   \
        if (e != cudaSuccess) return e;                                                                \
        k_multipoles_red_df<P><<<grid, threads, smem, s>>>(off, rel, C, rseg, rk, rcoef, Mr,          \
                                                           static_cast<dfl*>(Mrd), m002);              \
        break;                                                                                         \
    }
        NF_MP_RED_CASE(0)
        NF_MP_RED_CASE(1)
        NF_MP_RED_CASE(2)
        NF_MP_RED_CASE(3)
        NF_MP_RED_CASE(4)
        NF_MP_RED_CASE(5)
        NF_MP_RED_CASE(6)
        NF_MP_RED_CASE(7)
        NF_MP_RED_CASE(8)
        NF_MP_RED_CASE(9)
        NF_MP_RED_CASE(10)
        NF_MP_RED_CASE(11)
        NF_MP_RED_CASE(12)
#undef NF_MP_RED_CASE
        default:
            return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_taylor_forces_df(int p, const int* cell, const float4* rel, const void* Tdf, int N, int C,
                                    double scale, double* acc_far, float* acc_add, cudaStream_t s)
{
    const dfl* Td = static_cast<const dfl*>(Tdf);
    const int need = ((N + 1) / 2 + 127) / 128;
    const int grid = need < device_sms() * 16 ? need : device_sms() * 16;
    switch (p) {
#define NF_TAYLOR_DF_CASE(P)                                                                        \
    case P:                                                                                         \
        k_taylor_forces_df<P><<<grid, 128, 0, s>>>(cell, rel, Td, N, C, scale, acc_far, acc_add);   \
        break;
        NF_TAYLOR_DF_CASE(0)
        NF_TAYLOR_DF_CASE(1)
        NF_TAYLOR_DF_CASE(2)
        NF_TAYLOR_DF_CASE(3)
        NF_TAYLOR_DF_CASE(4)
        NF_TAYLOR_DF_CASE(5)
        NF_TAYLOR_DF_CASE(6)
        NF_TAYLOR_DF_CASE(7)
        NF_TAYLOR_DF_CASE(8)
        NF_TAYLOR_DF_CASE(9)
        NF_TAYLOR_DF_CASE(10)
        NF_TAYLOR_DF_CASE(11)
        NF_TAYLOR_DF_CASE(12)
#undef NF_TAYLOR_DF_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_unscale_taylors(const double* Tc, int C, int p, double w, double* T, cudaStream_t s)
{
    const int nt = far_terms(p);
    const long long total = (long long)C * nt;
    long long blocks = (total + 255) / 256;
    const long long cap = (long long)device_sms() * 16;
    if (blocks > cap) blocks = cap;
    k_unscale_taylors<<<(int)blocks, 256, 0, s>>>(Tc, total, nt, p, 1.0 / w, T);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_far_reduce(const double* M, int C, int nt, int nr, const int* seg, const int* kidx,
                              const double* coef, double* Mr, cudaStream_t s)
{
    const long long total = (long long)C * nr;
    long long blocks = (total + 255) / 256;
    const long long cap = (long long)device_sms() * 32;
    if (blocks > cap) blocks = cap;
    k_far_reduce<<<(int)blocks, 256, 0, s>>>(M, C, nt, nr, seg, kidx, coef, Mr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_far_sum_term(const double* M, int C, int nt, int term, double* partial, cudaStream_t s)
{
    k_far_sum_term<<<kSumBlocks, 256, 0, s>>>(M, C, nt, term, partial);
    count_launches(1);
    return cudaGetLastError();
}

int far_sum_partials() { return kSumBlocks; }

cudaError_t launch_far_rebuild(const void* Tr, bool df_in, int C, int p, int nt, int nr, const int4* ops,
                               const double2* opf, int t002, double lap, double t0_per_s002, const double* partial,
                               double* T, void* Tdf, cudaStream_t s)
{
    if (!T && !Tdf) return cudaSuccess;
    const void* fn;
    if (df_in)
        fn = T && Tdf ? (const void*)k_far_rebuild<true, true, true>
             : T      ? (const void*)k_far_rebuild<true, false, true>
                      : (const void*)k_far_rebuild<false, true, true>;
    else
        fn = T && Tdf ? (const void*)k_far_rebuild<true, true, false>
             : T      ? (const void*)k_far_rebuild<true, false, false>
                      : (const void*)k_far_rebuild<false, true, false>;
    const int slots = (T ? 1 : 0) + (Tdf ? 1 : 0);
    const size_t smem = (size_t)nt * (sizeof(int4) + sizeof(double2) + sizeof(float4)) +
                        (16 + (size_t)((nr + 3) & ~3)) * sizeof(int) + (size_t)kRebuildWarps * slots * nt * sizeof(double);
    cudaError_t e = ensure_smem(fn, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRebuildWarps * 32, smem);
    if (e != cudaSuccess) return e;
    long long blocks = ((long long)C + kRebuildWarps - 1) / kRebuildWarps;  // one warp per cell
    const long long cap = (long long)device_sms() * (per_sm > 0 ? per_sm : 1);  // one wave, all resident
    if (blocks > cap) blocks = cap;
    dfl* td = static_cast<dfl*>(Tdf);
#define NF_REBUILD_LAUNCH(A, B, D)                                                                           \
    k_far_rebuild<A, B, D><<<(int)blocks, kRebuildWarps * 32, smem, s>>>(Tr, C, p, nt, nr, ops, opf, t002, lap, \
                                                                        t0_per_s002, partial, T, td)
    if (df_in) {
        if (T && Tdf)
            NF_REBUILD_LAUNCH(true, true, true);
        else if (T)
            NF_REBUILD_LAUNCH(true, false, true);
        else
            NF_REBUILD_LAUNCH(false, true, true);
    } else {
        if (T && Tdf)
            NF_REBUILD_LAUNCH(true, true, false);
        else if (T)
            NF_REBUILD_LAUNCH(true, false, false);
        else
            NF_REBUILD_LAUNCH(false, true, false);
    }
#undef NF_REBUILD_LAUNCH
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_deriv_header(const DerivHeader& h, void* dst, cudaStream_t s)
{
    k_deriv_header<<<1, 32, 0, s>>>(h, static_cast<DerivHeader*>(dst));
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_far_contract(int K, int nout, const int* seg, const FarPair* pairs, const double* Dr,
                                const double2* Mh, double2* Th, cudaStream_t s)
{
    const long long nq = (long long)K * K * (K / 2 + 1);
    long long blocks = (nq * nout + 255) / 256;
    const long long cap = (long long)device_sms() * 64;
    if (blocks > cap) blocks = cap;
    const double scale = 1.0 / ((double)K * K * K);  // the unnormalised inverse transform
    k_far_contract<<<(int)blocks, 256, 0, s>>>(nq, nout, seg, pairs, Dr, Mh, Th, scale);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_taylor_forces(int p, const int* off, const float4* rel, const double* T, int N, int C, double w,
                                 double mass, double* acc_far, float* acc_add, cudaStream_t s)
{
    const int need = (N + 127) / 128;
    const int grid = need < device_sms() * 16 ? need : device_sms() * 16;
    switch (p) {
#define NF_TAYLOR_CASE(P)                                                                           \
    case P:                                                                                         \
        k_taylor_forces<P><<<grid, 128, 0, s>>>(off, rel, T, N, C, w, mass, acc_far, acc_add);      \
        break;
        NF_TAYLOR_CASE(0)
        NF_TAYLOR_CASE(1)
        NF_TAYLOR_CASE(2)
        NF_TAYLOR_CASE(3)
        NF_TAYLOR_CASE(4)
        NF_TAYLOR_CASE(5)
        NF_TAYLOR_CASE(6)
        NF_TAYLOR_CASE(7)
        NF_TAYLOR_CASE(8)
        NF_TAYLOR_CASE(9)
        NF_TAYLOR_CASE(10)
        NF_TAYLOR_CASE(11)
        NF_TAYLOR_CASE(12)
#undef NF_TAYLOR_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nf
