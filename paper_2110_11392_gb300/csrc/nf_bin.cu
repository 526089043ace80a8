// Binning: cell ids, cell offsets, stable LSD radix sort, cell-centred offsets.
//
// The paper stores particles in grid order with FP32 positions relative to
// the cell centre (Sec. "Force Accuracy", overview) on a K^3 grid of cells
// (Sec. "Two-Stage Execution").  Here the grid order comes from a stable sort
// by cell id done on the GPU:
//   k_shift      FP64 shift of every coordinate into cell units, cell id, and
//                an atomic histogram of cells (counts are order-independent);
//   scan         exclusive prefix sum -> cell_offsets;
//   radix passes stable LSD radix sort of (cell id, particle) with <= 2048
//                bins per pass: per-tile histograms, a scan of the
//                (bin, tile) matrix, then a stable scatter in which each warp
//                ranks its own elements in order with __match_any_sync;
//   k_rel        recomputes each sorted particle's offsets from its position.
// The FP64 shift uses explicitly rounded intrinsics so that no FMA
// contraction changes the rounding: the result is bit-identical to the plain
// CPU definition (t = x * (K/box), c = floor(t), offset = fp32((t - c) - 1/2),
// cell = c mod K).
#include <cuda_runtime.h>

#include <cstdio>

#include "nf_internal.cuh"

namespace nf {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int find_box(const BoxDev* boxes, int nboxes, int e)
{
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].part_base <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One coordinate into cell units, in FP64 as defined: t = x * kl, c = floor(t),
// offset = fp32((t - c) - 1/2), cell = c mod K.  Returns the cell, writes the
// offset; flags non-finite input.
__device__ __forceinline__ int cell_coord_fp64(float x, double kl, int K, float* off, bool* bad)
{
    double xd = (double)x;
    if (!isfinite(xd)) {
        *bad = true;
        *off = 0.0f;
        return 0;
    }
    double t = __dmul_rn(xd, kl);
    double c = floor(t);
    double frac = __dsub_rn(t, c);
    double o = __dsub_rn(frac, 0.5);
    *off = __double2float_rn(o);
    // c mod K into [0, K): c is an exact integer, so integer arithmetic gives
    // the same value as an FP64 remainder (and avoids the slow FP64 one)
    if (fabs(c) < 2147483647.0) {
        int cm = (int)c % K;
        return cm < 0 ? cm + K : cm;
    }
    double cm = fmod(c, (double)K);
    if (cm < 0.0) cm = __dadd_rn(cm, (double)K);
    return (int)cm;
}

// The same function in integer arithmetic, used when kl = kl_mant * 2^kl_exp
// with a short odd mantissa (the unit box: kl = K).  Then t = x * kl, floor(t),
// t - c and (t - c) - 1/2 are all exact in FP64 for 2^-29 <= |x| < 2^30, so the
// FP64 definition reduces to one rounding of an exact value, which this path
// computes with 64-bit integers (the GPU's FP64 pipe is slow).  Other inputs
// take the FP64 path; both give identical results.
__device__ __forceinline__ int cell_coord(float x, const BoxDev& B, float* off, bool* bad)
{
    const unsigned bits = __float_as_uint(x);
    const int E = (int)((bits >> 23) & 0xFF);
    if (B.kl_mant > 0 && E >= 127 - 29 && E < 127 + 30) {
        const long long P = (long long)((bits & 0x7FFFFFu) | 0x800000u) * (long long)B.kl_mant;
        const int s = 150 - E - B.kl_exp;  // t = +-P * 2^-s
        if (s >= 1 && s <= 53) {
            const long long one = 1LL << s;
            const long long low = P & (one - 1);
            long long c;
            long long frac;  // (t - c) * 2^s, in [0, 2^s)
            if ((int)(bits >> 31) == 0) {
                c = P >> s;
                frac = low;
            } else {
                c = -(P >> s) - (low != 0);
                frac = low ? one - low : 0;
            }
            const long long o = frac - (one >> 1);
            // exact scaling of the rounded integer by 2^-s
            *off = __ll2float_rn(o) * __int_as_float((127 - s) << 23);
            long long cm = c % B.K;
            return (int)(cm < 0 ? cm + B.K : cm);
        }
    }
    return cell_coord_fp64(x, B.kl, B.K, off, bad);
}

__global__ void k_fill_boxes(BoxFill f, BoxDev* boxes)
{
    int i = threadIdx.x;
    if (i < f.count) boxes[f.first + i] = f.b[i];
}

__global__ void k_shift(const float* __restrict__ pos, int Ntot, const BoxDev* __restrict__ boxes,
                        int nboxes, int* __restrict__ keys, int* __restrict__ counts,
                        WsHeader* hdr)
{
    bool bad = false;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ntot; e += gridDim.x * blockDim.x) {
        const BoxDev& B = boxes[find_box(boxes, nboxes, e)];
        float o;
        int cx = cell_coord(pos[3 * (size_t)e + 0], B, &o, &bad);
        int cy = cell_coord(pos[3 * (size_t)e + 1], B, &o, &bad);
        int cz = cell_coord(pos[3 * (size_t)e + 2], B, &o, &bad);
        int key = B.cell_base + (cx * B.K + cy) * B.K + cz;
        keys[e] = key;
        atomicAdd(&counts[key], 1);
    }
    if (bad) atomicOr(&hdr->status, 1 << NF_ERR_NONFINITE);
}

__global__ void k_rel(const float* __restrict__ pos, int Ntot, const BoxDev* __restrict__ boxes,
                      int nboxes, const int* __restrict__ perm, float4* __restrict__ rel)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < Ntot; s += gridDim.x * blockDim.x) {
        int e = perm[s];
        const BoxDev& B = boxes[find_box(boxes, nboxes, e)];
        bool bad = false;
        float4 r;
        cell_coord(pos[3 * (size_t)e + 0], B, &r.x, &bad);
        cell_coord(pos[3 * (size_t)e + 1], B, &r.y, &bad);
        cell_coord(pos[3 * (size_t)e + 2], B, &r.z, &bad);
        r.w = __int_as_float(e);
        rel[s] = r;
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 (reduce, scan of block sums, apply)
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

// Exclusive prefix of v over the block; *total gets the block sum.
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* total)
{
    __shared__ unsigned warp_sum[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[w] = x;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        unsigned s = lane < nw ? warp_sum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        warp_sum[lane] = s;  // inclusive
    }
    __syncthreads();
    unsigned before = (w > 0 ? warp_sum[w - 1] : 0u) + (x - v);
    *total = warp_sum[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void k_scan_reduce(const unsigned* __restrict__ d, size_t n, unsigned* __restrict__ aux)
{
    size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanPer;
    unsigned s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < n) s += d[base + i];
    unsigned total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) aux[blockIdx.x] = total;
}

__global__ void k_scan_aux(unsigned* aux, size_t nb)
{
    unsigned carry = 0;
    for (size_t base = 0; base < nb; base += kScanTile) {
        size_t i0 = base + (size_t)threadIdx.x * kScanPer;
        unsigned v[kScanPer];
        unsigned s = 0;
#pragma unroll
        for (int i = 0; i < kScanPer; ++i) {
            v[i] = (i0 + i < nb) ? aux[i0 + i] : 0u;
            s += v[i];
        }
        unsigned total;
        unsigned pre = block_excl_scan(s, &total) + carry;
#pragma unroll
        for (int i = 0; i < kScanPer; ++i) {
            if (i0 + i < nb) aux[i0 + i] = pre;
            pre += v[i];
        }
        carry += total;
    }
}

__global__ void k_scan_apply(unsigned* __restrict__ d, size_t n, const unsigned* __restrict__ aux)
{
    size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanPer;
    unsigned v[kScanPer];
    unsigned s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = (base + i < n) ? d[base + i] : 0u;
        s += v[i];
    }
    unsigned total;
    unsigned pre = block_excl_scan(s, &total) + aux[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < n) d[base + i] = pre;
        pre += v[i];
    }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort
// ---------------------------------------------------------------------------

constexpr int kRxWarps = 8;
constexpr int kRxMaxRounds = 64;            // rounds of 32 elements per warp (upper bound)
constexpr int kRxMaxBits = 11;

__global__ void __launch_bounds__(kRxWarps * 32)
k_radix_up(const int* __restrict__ keys, int N, int shift, int mask, int bins, int tiles, int rounds,
           unsigned* __restrict__ H)
{
    extern __shared__ unsigned hist[];
    for (int b = threadIdx.x; b < bins; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const int tile = kRxWarps * 32 * rounds;
    size_t base = (size_t)blockIdx.x * tile;
#pragma unroll 4
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
        size_t e = base + i;
        if (e < (size_t)N) atomicAdd(&hist[(keys[e] >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < bins; b += blockDim.x)
        H[(size_t)b * tiles + blockIdx.x] = hist[b];
}

// Stable scatter of one tile.  vals_in == nullptr means "value = index".
// keys_out == nullptr skips the key write (last pass).
__global__ void __launch_bounds__(kRxWarps * 32)
k_radix_down(const int* __restrict__ keys_in, const int* __restrict__ vals_in, int N, int shift,
             int mask, int bins, int tiles, int rounds, const unsigned* __restrict__ H,
             int* __restrict__ keys_out, int* __restrict__ vals_out)
{
    extern __shared__ unsigned cnt[];  // [kRxWarps][bins]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRxWarps * bins; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const size_t sub = (size_t)blockIdx.x * (kRxWarps * 32 * rounds) + (size_t)w * (32 * rounds);
    unsigned* my = cnt + w * bins;
    const unsigned lt = (1u << lane) - 1u;
    // counts of this warp's sub-tile; keys are loaded four rounds at a time so
    // the loads overlap (rounds is a multiple of 4)
    constexpr int G = 4;
    for (int r0 = 0; r0 < rounds; r0 += G) {
        if (sub + (size_t)r0 * 32 >= (size_t)N) break;
        int kv[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const size_t e = sub + (size_t)(r0 + g) * 32 + lane;
            kv[g] = e < (size_t)N ? keys_in[e] : -1;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const bool valid = kv[g] >= 0;
            const int d = valid ? ((kv[g] >> shift) & mask) : bins;
            const unsigned peers = __match_any_sync(kFull, d);
            if (valid && lane == __ffs(peers) - 1) my[d] += __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    // global offsets: bins of earlier tiles and earlier warps of this tile
    for (int b = threadIdx.x; b < bins; b += blockDim.x) {
        unsigned run = H[(size_t)b * tiles + blockIdx.x];
        for (int q = 0; q < kRxWarps; ++q) {
            unsigned c = cnt[q * bins + b];
            cnt[q * bins + b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int r0 = 0; r0 < rounds; r0 += G) {
        if (sub + (size_t)r0 * 32 >= (size_t)N) break;
        int kv[G], vv[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const size_t e = sub + (size_t)(r0 + g) * 32 + lane;
            const bool valid = e < (size_t)N;
            kv[g] = valid ? keys_in[e] : -1;
            vv[g] = valid ? (vals_in ? vals_in[e] : (int)e) : 0;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const bool valid = kv[g] >= 0;
            const int d = valid ? ((kv[g] >> shift) & mask) : bins;
            const unsigned peers = __match_any_sync(kFull, d);
            const unsigned base = valid ? my[d] : 0u;
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) my[d] = base + __popc(peers);
            __syncwarp();
            if (valid) {
                const unsigned p = base + __popc(peers & lt);
                if (keys_out) keys_out[p] = kv[g];
                vals_out[p] = vv[g];
            }
        }
    }
}

int grid_for(size_t n, int threads)
{
    size_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535ull * 16) b = 65535ull * 16;
    return (int)b;
}

}  // namespace

cudaError_t launch_fill_boxes(const BoxFill& f, BoxDev* boxes, cudaStream_t s)
{
    k_fill_boxes<<<1, kMaxBoxesPerFill, 0, s>>>(f, boxes);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_shift(const float* pos, int Ntot, const BoxDev* boxes, int nboxes, int* keys,
                         int* counts, WsHeader* hdr, cudaStream_t s)
{
    k_shift<<<grid_for(Ntot, 256), 256, 0, s>>>(pos, Ntot, boxes, nboxes, keys, counts, hdr);
    count_launches(1);
    return cudaGetLastError();
}

size_t scan_aux_words(size_t n)
{
    return (n + kScanTile - 1) / kScanTile + 1;
}

cudaError_t launch_scan(unsigned* data, size_t n, unsigned* aux, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    size_t nb = (n + kScanTile - 1) / kScanTile;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, aux);
    k_scan_aux<<<1, kScanThreads, 0, s>>>(aux, nb);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, aux);
    count_launches(3);
    return cudaGetLastError();
}

RadixPlan radix_plan(int64_t N, int64_t C)
{
    int bits = 1;
    while ((int64_t(1) << bits) < C) ++bits;
    RadixPlan p;
    p.passes = (bits + kRxMaxBits - 1) / kRxMaxBits;
    p.digit_bits = (bits + p.passes - 1) / p.passes;
    p.bins = 1 << p.digit_bits;
    // Enough tiles to fill every SM several times over (the rounds of a warp
    // run one after another), but no more than the (bin, tile) matrix needs.
    p.rounds = kRxMaxRounds;
    while (p.rounds > 4 && (N + kRxWarps * 32 * p.rounds - 1) / (kRxWarps * 32 * p.rounds) < 1024) p.rounds >>= 1;
    const int64_t tile = (int64_t)kRxWarps * 32 * p.rounds;
    p.tiles = (int)((N + tile - 1) / tile);
    if (p.tiles < 1) p.tiles = 1;
    return p;
}

size_t radix_hist_words(const RadixPlan& p)
{
    return (size_t)p.bins * p.tiles;
}

cudaError_t radix_sort(const RadixPlan& p, int N, int* keys_a, int* keys_b, int* vals_a,
                       int* vals_b, int* perm, unsigned* hist, unsigned* aux, cudaStream_t s)
{
    const size_t smem_up = (size_t)p.bins * sizeof(unsigned);
    const size_t smem_down = (size_t)kRxWarps * p.bins * sizeof(unsigned);
    cudaError_t err = ensure_smem((const void*)k_radix_down, (int)smem_down);
    if (err != cudaSuccess) return err;
    const int* kin = keys_a;
    const int* vin = nullptr;
    int* kbuf[2] = {keys_b, keys_a};
    int* vbuf[2] = {vals_b, vals_a};
    for (int pass = 0; pass < p.passes; ++pass) {
        const int shift = pass * p.digit_bits;
        const int mask = p.bins - 1;
        const bool last = pass == p.passes - 1;
        int* kout = last ? nullptr : kbuf[pass & 1];
        int* vout = last ? perm : vbuf[pass & 1];
        k_radix_up<<<p.tiles, kRxWarps * 32, smem_up, s>>>(kin, N, shift, mask, p.bins, p.tiles, p.rounds, hist);
        count_launches(1);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if ((err = launch_scan(hist, radix_hist_words(p), aux, s)) != cudaSuccess) return err;
        k_radix_down<<<p.tiles, kRxWarps * 32, smem_down, s>>>(kin, vin, N, shift, mask, p.bins,
                                                               p.tiles, p.rounds, hist, kout, vout);
        count_launches(1);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        kin = kout;
        vin = vout;
    }
    return cudaSuccess;
}

cudaError_t launch_rel(const float* pos, int Ntot, const BoxDev* boxes, int nboxes,
                       const int* perm, float4* rel, cudaStream_t s)
{
    k_rel<<<grid_for(Ntot, 256), 256, 0, s>>>(pos, Ntot, boxes, nboxes, perm, rel);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nf
