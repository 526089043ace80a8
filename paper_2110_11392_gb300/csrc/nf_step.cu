// Time stepping on the device: Kick-Drift-Kick leapfrog and the global time
// step of Eq. (timestep) (Sec. "Time Stepping").
//
//   k_kick         v += a * (dt * factor)
//   k_drift        x = wrap(x + v dt) into [0, box)
//   k_cell_ratio   per occupied cell: v_rms (without subtracting the cell's
//                  mean velocity, as the paper specifies) and a_max, from the
//                  binning of the last force call; the smallest v_rms / a_max
//                  over cells (atomic min on the bits of a positive float);
//                  per-block FP64 sums of |v|^2 and the largest |a|
//   k_timestep     dt = min(eta_H / H, eta_acc * max(min_c ratio, global ratio))
// dt lives in device memory so a whole step (and a loop of steps) can run
// without the host and be captured in a CUDA graph.
#include <cuda_runtime.h>

#include "nf_internal.cuh"

namespace nf {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__global__ void k_kick(float* __restrict__ vel, const float* __restrict__ acc, int n3, const double* dt,
                       double factor)
{
    const float h = (float)(*dt * factor);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x)
        vel[i] = fmaf(acc[i], h, vel[i]);
}

__global__ void k_drift(float* __restrict__ pos, const float* __restrict__ vel, int n3, const double* dt,
                        float box)
{
    const float h = (float)*dt;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) {
        float x = fmaf(vel[i], h, pos[i]);
        x -= box * floorf(x / box);
        if (x >= box) x -= box;
        if (x < 0.0f) x = 0.0f;
        pos[i] = x;
    }
}

__global__ void k_step_init(StepScratch* st)
{
    if (threadIdx.x == 0) {
        st->min_ratio_bits = 0x7f800000u;  // +inf
        st->max_a2_bits = 0u;
    }
}

__global__ void k_cell_ratio(const int* __restrict__ off, const int* __restrict__ perm,
                             const float* __restrict__ vel, const float* __restrict__ acc, int C,
                             StepScratch* st)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    float best = __int_as_float(0x7f800000);  // +inf
    double v2_sum = 0.0;
    float a2_max = 0.0f;
    for (int c = warp; c < C; c += nwarps) {
        const int s0 = off[c], s1 = off[c + 1];
        if (s1 == s0) continue;
        float v2 = 0.0f, a2 = 0.0f;
        for (int s = s0 + lane; s < s1; s += 32) {
            const int i = perm[s];
            const float vx = vel[3 * (size_t)i], vy = vel[3 * (size_t)i + 1], vz = vel[3 * (size_t)i + 2];
            const float ax = acc[3 * (size_t)i], ay = acc[3 * (size_t)i + 1], az = acc[3 * (size_t)i + 2];
            const float q = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
            v2 += q;
            v2_sum += (double)q;
            a2 = fmaxf(a2, fmaf(ax, ax, fmaf(ay, ay, az * az)));
        }
        for (int o = 16; o; o >>= 1) {
            v2 += __shfl_xor_sync(kFull, v2, o);
            a2 = fmaxf(a2, __shfl_xor_sync(kFull, a2, o));
        }
        a2_max = fmaxf(a2_max, a2);
        if (a2 > 0.0f) best = fminf(best, sqrtf(v2 / (float)(s1 - s0)) / sqrtf(a2));
    }
    // block reductions: min ratio, max |a|^2 (order-free), FP64 sum of |v|^2 in a fixed order
    __shared__ double red_v[32];
    __shared__ float red_b[32], red_a[32];
    for (int o = 16; o; o >>= 1) {
        v2_sum += __shfl_xor_sync(kFull, v2_sum, o);
        best = fminf(best, __shfl_xor_sync(kFull, best, o));
        a2_max = fmaxf(a2_max, __shfl_xor_sync(kFull, a2_max, o));
    }
    const int w = threadIdx.x >> 5;
    if (lane == 0) {
        red_v[w] = v2_sum;
        red_b[w] = best;
        red_a[w] = a2_max;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        float b = red_b[0], a = red_a[0];
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            v += red_v[q];
            b = fminf(b, red_b[q]);
            a = fmaxf(a, red_a[q]);
        }
        st->v2_block[blockIdx.x] = v;
        atomicMin(&st->min_ratio_bits, __float_as_uint(b));  // positive floats order like their bits
        atomicMax(&st->max_a2_bits, __float_as_uint(a));
    }
}

__global__ void k_timestep(StepScratch* st, int nblocks, long long N, double eta_acc, double eta_h, double hubble,
                           double* dt)
{
    if (threadIdx.x != 0) return;
    double v2 = 0.0;
    for (int b = 0; b < nblocks; ++b) v2 += st->v2_block[b];
    const double amax = sqrt((double)__uint_as_float(st->max_a2_bits));
    const double glob = amax > 0.0 ? sqrt(v2 / (double)N) / amax : __longlong_as_double(0x7ff0000000000000LL);
    const double cellmin = (double)__uint_as_float(st->min_ratio_bits);
    double r = fmax(cellmin, glob);
    double out = eta_acc * r;
    if (hubble > 0.0) out = fmin(out, eta_h / hubble);
    *dt = out;
}

int grid_for(size_t n, int threads)
{
    size_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535ull * 16) b = 65535ull * 16;
    return (int)b;
}

}  // namespace

cudaError_t launch_kick(float* vel, const float* acc, int N, const double* dt, double factor, cudaStream_t s)
{
    k_kick<<<grid_for(3 * (size_t)N, 256), 256, 0, s>>>(vel, acc, 3 * N, dt, factor);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_drift(float* pos, const float* vel, int N, const double* dt, float box, cudaStream_t s)
{
    k_drift<<<grid_for(3 * (size_t)N, 256), 256, 0, s>>>(pos, vel, 3 * N, dt, box);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_timestep(const int* off, const int* perm, const float* vel, const float* acc, int C, long long N,
                            double eta_acc, double eta_h, double hubble, StepScratch* st, double* dt, cudaStream_t s)
{
    k_step_init<<<1, 32, 0, s>>>(st);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_cell_ratio<<<kStepBlocks, 256, 0, s>>>(off, perm, vel, acc, C, st);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_timestep<<<1, 32, 0, s>>>(st, kStepBlocks, N, eta_acc, eta_h, hubble, dt);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nf
