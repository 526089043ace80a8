// Fused multiply-add throughput probe: the measured denominator beside the
// derived FP32 and FP64 peaks of the benchmark's rooflines.  A measurement aid
// of the benchmark, built into its own small library (libnf_probe.so), not part
// of libnf or of the paper's method.  Every thread runs kChains independent
// multiply-add chains (scalar FP32, packed .f32x2 pairs, or FP64) so the pipe,
// not latency, limits the rate.  The chain constants keep every value normal
// and finite: x -> x * 0.999 + 0.001 converges to 1.
#include <cuda_runtime.h>

#include <cstddef>

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

typedef unsigned long long p2;

__device__ __forceinline__ p2 pack2(float a, float b)
{
    p2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(p2 v, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ p2 ffma2(p2 a, p2 b, p2 c)
{
    p2 d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// MODE 0: scalar fma.rn.f32; 1: packed fma.rn.f32x2; 2: fma.rn.f64
template <int MODE>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(float* __restrict__ sink, int iters, float m, float a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float s = 0.0f;
    if constexpr (MODE == 1) {
        p2 x[kChains];
        const p2 mm = pack2(m, m), aa = pack2(a, a);
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = pack2(0.5f + 1e-3f * c, 0.25f + 1e-3f * t);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int c = 0; c < kChains; ++c) x[c] = ffma2(x[c], mm, aa);
            }
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float lo, hi;
            unpack2(x[c], lo, hi);
            s += lo + hi;
        }
    } else if constexpr (MODE == 2) {
        double x[kChains];
        const double md = (double)m, ad = (double)a;
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = 0.5 + 1e-3 * c + 1e-6 * t;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], md, ad);
            }
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += (float)x[c];
    } else {
        float x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = 0.5f + 1e-3f * c + 1e-6f * t;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], m, a);
            }
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += x[c];
    }
    sink[t] = s;
}

int probe_blocks()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * kProbeBlocksPerSm;
}

}  // namespace

extern "C" {

// Values the sink buffer must hold: one per thread of the launch.
size_t nfp_fma_probe_sink_floats(void) { return (size_t)probe_blocks() * kProbeThreads; }

// Launches the probe on `stream` (asynchronous).  mode 0: scalar fma.rn.f32,
// 1: packed fma.rn.f32x2, 2: fma.rn.f64.  *flop receives the floating-point
// operations of the launch (2 per multiply-add and lane).  Returns 0, 1 for a
// bad argument (NULL pointer, iters outside [1, 2^24], another mode), or 2 +
// the CUDA error code when the launch fails.
int nfp_fma_probe(float* sink, int iters, int mode, double* flop, cudaStream_t s)
{
    if (!sink || !flop || iters < 1 || iters > (1 << 24) || mode < 0 || mode > 2) return 1;
    const int blocks = probe_blocks();
    if (mode == 1)
        k_fma_probe<1><<<blocks, kProbeThreads, 0, s>>>(sink, iters, 0.999f, 0.001f);
    else if (mode == 2)
        k_fma_probe<2><<<blocks, kProbeThreads, 0, s>>>(sink, iters, 0.999f, 0.001f);
    else
        k_fma_probe<0><<<blocks, kProbeThreads, 0, s>>>(sink, iters, 0.999f, 0.001f);
    // lanes x multiply-adds per lane x 2 flop
    *flop = (double)blocks * kProbeThreads * iters * kUnroll * kChains * (mode == 1 ? 2 : 1) * 2.0;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : 2 + (int)e;
}

}  // extern "C"
