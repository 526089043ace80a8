// Cell multipoles in the complete basis, Eq. (multipoles) (Sec. "Computation
// of the Cell Multipoles"):
//     M^{abc}_cell = sum over the cell's particles of x^a y^b z^c,
//     0 <= a <= p, 0 <= b <= p - a, 0 <= c <= p - a - b,
// with (x, y, z) the displacement from the cell centre in box units.
// The paper evaluates these on CPU cores in FP64 with unrolled, interleaved
// SIMD loops; here one block takes one cell and one thread one term (a, b, c).
// The particles of the cell (contiguous after binning) are taken 64 at a time:
// threads first build the powers x^0..x^p, y^0..y^p, z^0..z^p of every particle
// of the chunk in shared memory (one thread per particle and axis) and the
// products x^a y^b (one per particle and (a, b) pair, the paper's
// precomputation that turns the innermost update into an FMA), then every term
// thread accumulates (x^a y^b) * z^c with one FMA per particle.
// Arithmetic is FP64 throughout, as the paper keeps its far-field internals.
#include <cuda_runtime.h>

#include "nf_internal.cuh"

namespace nf {

namespace {

constexpr int kChunk = 64;

__global__ void k_multipoles(const int* __restrict__ off, const float4* __restrict__ rel, int C, double w, int p,
                             int nterms, double* __restrict__ M)
{
    // shared: powers [3][kChunk][p + 1], then x^a y^b products [kChunk][nab]
    extern __shared__ double pw[];
    const int P1 = p + 1;
    const int nab = (p + 1) * (p + 2) / 2;
    double* XY = pw + (size_t)3 * kChunk * P1;
    // decode this thread's (a, b, c) from its term index, in the output order
    int a = 0, b = 0, c = 0;
    const int t = threadIdx.x;
    if (t < nterms) {
        int r = t;
        for (a = 0; a <= p; ++a) {
            const int n_a = (p - a + 1) * (p - a + 2) / 2;  // terms with this a
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
    // index of (a, b) among the pairs a = 0..p, b = 0..p-a
    const int ab = a * (p + 1) - a * (a - 1) / 2 + b;
    for (int cell = blockIdx.x; cell < C; cell += gridDim.x) {
        const int s0 = off[cell], s1 = off[cell + 1];
        double acc = 0.0;
        for (int q0 = s0; q0 < s1; q0 += kChunk) {
            const int nq = min(kChunk, s1 - q0);
            __syncthreads();
            for (int i = threadIdx.x; i < 3 * nq; i += blockDim.x) {
                const int q = i / 3, d = i - 3 * q;
                const float4 r4 = rel[q0 + q];
                const double x = (double)(d == 0 ? r4.x : (d == 1 ? r4.y : r4.z)) * w;
                double* row = pw + ((size_t)d * kChunk + q) * P1;
                double v = 1.0;
                row[0] = 1.0;
                for (int e = 1; e <= p; ++e) {
                    v *= x;
                    row[e] = v;
                }
            }
            __syncthreads();
            // x^a y^b once per particle and (a, b) pair
            for (int i = threadIdx.x; i < nq * nab; i += blockDim.x) {
                const int q = i / nab, k = i - q * nab;
                int aa = 0, kk = k;
                while (kk > p - aa) {
                    kk -= p - aa + 1;
                    ++aa;
                }
                XY[(size_t)q * nab + k] = pw[(size_t)q * P1 + aa] * pw[((size_t)kChunk + q) * P1 + kk];
            }
            __syncthreads();
            if (t < nterms) {
                const double* Z = pw + (size_t)2 * kChunk * P1;
                for (int q = 0; q < nq; ++q) acc = fma(XY[(size_t)q * nab + ab], Z[q * P1 + c], acc);
            }
        }
        if (t < nterms) M[(size_t)cell * nterms + t] = acc;
    }
}

}  // namespace

int multipole_terms(int p) { return (p + 3) * (p + 2) * (p + 1) / 6; }

cudaError_t launch_multipoles(const int* off, const float4* rel, int C, double w, int p, double* M, cudaStream_t s)
{
    const int nterms = multipole_terms(p);
    const int threads = ((nterms + 31) / 32) * 32;
    const size_t smem = ((size_t)3 * kChunk * (p + 1) + (size_t)kChunk * (p + 1) * (p + 2) / 2) * sizeof(double);
    cudaError_t e = ensure_smem((const void*)k_multipoles, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = C < sms * 32 ? C : sms * 32;
    k_multipoles<<<grid, threads, smem, s>>>(off, rel, C, w, p, nterms, M);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nf
