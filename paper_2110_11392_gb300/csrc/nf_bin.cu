// Binning: cell ids, cell offsets and cell-centred offsets in grid order.
//
// The paper stores particles in grid order with FP32 positions relative to
// the cell centre (Sec. "Force Accuracy", overview) on a K^3 grid of cells
// (Sec. "Two-Stage Execution").  Here the grid order comes from a stable
// least-significant-digit sort of (cell id, particle) done on the GPU, with
// digits of at most 9 bits (one pass for K <= 8, two for K <= 32, three for
// K <= 128):
//   k_tile_hist  per tile of 2048 particles, the count of every digit value
//                of this pass (the first pass computes the cell ids from the
//                positions, FP64 rule below; later ones read them), written
//                digit-major so that one exclusive scan of the whole matrix
//                gives every (digit, tile) run its first output slot;
//   scan         that exclusive scan (reduce, scan of block sums, apply);
//   k_sort_pass  one stable pass over the same tiles: the first pass computes
//                each particle's cell id and cell-centred offsets from its
//                position, later passes read them back; a tile ranks its
//                particles by digit in input order (each warp ranks its own
//                consecutive elements, finding the lanes with the same digit
//                by one vote per digit bit), reorders the tile in shared
//                memory and writes every run contiguously.  The
//                offsets travel with the particle (float4, .w = original
//                index), so no pass gathers positions at random;
//   k_cell_off   cell_offsets from the sorted cell ids (the first slot of
//                every cell; empty cells get the next cell's first slot).
// The FP64 shift uses explicitly rounded intrinsics so that no FMA
// contraction changes the rounding: the result is bit-identical to the plain
// CPU definition (t = x * (K/box), c = floor(t), offset = fp32((t - c) - 1/2),
// cell = c mod K).
#include <cuda_runtime.h>

#include <algorithm>
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
    if (c >= 0.0 && c < (double)K) return (int)c;  // inside the box: no wrap
    if (fabs(c) < 2147483647.0) {
        int cm = (int)c % K;
        return cm < 0 ? cm + K : cm;
    }
    double cm = fmod(c, (double)K);
    if (cm < 0.0) cm = __dadd_rn(cm, (double)K);
    return (int)cm;
}

struct CellCoord {
    int c;      // cell index in [0, K)
    float off;  // cell-centred offset
    int bad;    // non-finite input
};

// The same function for any K / box and any x.  In integer arithmetic when
// kl = kl_mant * 2^kl_exp with a short odd mantissa (the unit box: kl = K):
// then t = x * kl, floor(t), t - c and (t - c) - 1/2 are all exact in FP64 for
// 2^-29 <= |x| < 2^30, so the FP64 definition reduces to one rounding of an
// exact value, which this path computes with 64-bit integers (the GPU's FP64
// pipe is slow).  Other inputs take the FP64 path; both give identical
// results.  Out of line: the sort passes inline only the power-of-two path of
// cell_coord, which keeps their code (24 coordinates per thread) small.
#ifndef NF_BIN_SLOW_NOINLINE
#define NF_BIN_SLOW_NOINLINE 1
#endif
#if NF_BIN_SLOW_NOINLINE
__device__ __noinline__
#else
__device__ __forceinline__
#endif
CellCoord cell_coord_general(float x, int K, int kl_mant, int kl_exp, double kl)
{
    CellCoord r;
    r.bad = 0;
    const unsigned bits = __float_as_uint(x);
    const int E = (int)((bits >> 23) & 0xFF);
    if (kl_mant > 0 && E >= 127 - 29 && E < 127 + 30) {
        const long long P = (long long)((bits & 0x7FFFFFu) | 0x800000u) * (long long)kl_mant;
        const int s = 150 - E - kl_exp;  // t = +-P * 2^-s
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
            r.off = __ll2float_rn(o) * __int_as_float((127 - s) << 23);
            if (c >= 0 && c < K) {  // inside the box: no wrap (64-bit % is slow)
                r.c = (int)c;
                return r;
            }
            long long cm = c % K;
            r.c = (int)(cm < 0 ? cm + K : cm);
            return r;
        }
    }
    bool bad = false;
    r.c = cell_coord_fp64(x, kl, K, &r.off, &bad);
    r.bad = bad;
    return r;
}

__device__ __forceinline__ int cell_coord(float x, const BoxDev& B, float* off, bool* bad)
{
    // K / box a power of two and x >= 0: t = x * K/box is exact in FP32 as in
    // FP64, so are c = floor(t) and t - c (for t >= 0), and one FP32
    // subtraction rounds (t - c) - 1/2 exactly as the FP64 rule's final
    // rounding does.  (For t < 0, t - floor(t) can round in FP32.)
    if (B.kl_pow2 != 0.0f) {
        const float t = __fmul_rn(x, B.kl_pow2);
        if (t >= 0.0f && t < 1073741824.0f) {  // false for NaN
            const float c = floorf(t);
            *off = __fsub_rn(__fsub_rn(t, c), 0.5f);
            const int ci = (int)c;
            if (ci < B.K) return ci;
            return ci % B.K;
        }
    }
    const CellCoord r = cell_coord_general(x, B.K, B.kl_mant, B.kl_exp, B.kl);
    *off = r.off;
    if (r.bad) *bad = true;
    return r.c;
}

__global__ void k_fill_boxes(BoxFill f, BoxDev* boxes)
{
    int i = threadIdx.x;
    if (i < f.count) boxes[f.first + i] = f.b[i];
}

// Cell id (global: cell_base + local id) and cell-centred offsets of particle
// e, whose coordinates are x[0..2].
__device__ __forceinline__ int particle_key(const float* x, int e, const BoxDev* __restrict__ boxes, int nboxes,
                                           float4* rel, bool* bad)
{
    const BoxDev& B = boxes[nboxes > 1 ? find_box(boxes, nboxes, e) : 0];
    float4 r;
    const int cx = cell_coord(x[0], B, &r.x, bad);
    const int cy = cell_coord(x[1], B, &r.y, bad);
    const int cz = cell_coord(x[2], B, &r.z, bad);
    r.w = __int_as_float(e);
    *rel = r;
    return B.cell_base + (cx * B.K + cy) * B.K + cz;
}

// Copies the coordinates of particles [base, base + n) into shared memory
// (3n floats) with coalesced loads, 16 bytes at a time when aligned.  A full
// tile issues all of a thread's loads before its first store, so their
// latencies overlap instead of adding up.
__device__ __forceinline__ void stage_positions(const float* __restrict__ pos, size_t base, int n, float* spos)
{
    const float* src = pos + 3 * base;
    const int nf = 3 * n;
    constexpr int kPer = 3 * kSortTile / 4 / (kSortWarps * 32);
    static_assert(kPer * 4 * kSortWarps * 32 == 3 * kSortTile, "a tile's coordinates split evenly into float4s");
    if (n == kSortTile && (reinterpret_cast<uintptr_t>(src) & 15) == 0 && blockDim.x == kSortWarps * 32) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
        float4* d4 = reinterpret_cast<float4*>(spos);
        float4 t[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) t[r] = s4[r * kSortWarps * 32 + threadIdx.x];
#pragma unroll
        for (int r = 0; r < kPer; ++r) d4[r * kSortWarps * 32 + threadIdx.x] = t[r];
    } else if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const int n4 = nf >> 2;
        const float4* s4 = reinterpret_cast<const float4*>(src);
        float4* d4 = reinterpret_cast<float4*>(spos);
        for (int i = threadIdx.x; i < n4; i += blockDim.x) d4[i] = s4[i];
        for (int i = 4 * n4 + threadIdx.x; i < nf; i += blockDim.x) spos[i] = src[i];
    } else {
        for (int i = threadIdx.x; i < nf; i += blockDim.x) spos[i] = src[i];
    }
}

// One warp copies the coordinates of its own particles [base, base + n),
// n <= 32 * kWarpElems, into shared memory (3n floats) with coalesced loads,
// all of a lane's loads issued before its first store.  Only this warp reads
// them back, so a __syncwarp orders the copy (no block-wide barrier).
constexpr int kWarpElems = kSortTile / (kSortWarps * 32);  // elements per lane
__device__ __forceinline__ void stage_positions_warp(const float* __restrict__ pos, size_t base, int n,
                                                     float* spos, int lane)
{
    const float* src = pos + 3 * base;
    constexpr int kPer = 3 * kWarpElems * 32 / 4 / 32;  // float4 per lane for a full warp share
    static_assert(kPer * 4 * 32 == 3 * kWarpElems * 32, "a warp's coordinates split evenly into float4s");
    if (n == 32 * kWarpElems && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
        float4* d4 = reinterpret_cast<float4*>(spos);
        float4 t[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) t[r] = s4[r * 32 + lane];
#pragma unroll
        for (int r = 0; r < kPer; ++r) d4[r * 32 + lane] = t[r];
    } else {
        for (int i = lane; i < 3 * n; i += 32) spos[i] = src[i];
    }
    __syncwarp();
}

// Counts of every digit value in each tile, written to M[digit * tiles + tile].
// FIRST computes the cell ids from the positions (and flags non-finite input).
template <bool FIRST>
__global__ void __launch_bounds__(kSortWarps * 32)
k_tile_hist(const float* __restrict__ pos, const BoxDev* __restrict__ boxes, int nboxes,
            const int* __restrict__ key_in, int N, int shift, int bits, int tiles, unsigned* __restrict__ M,
            WsHeader* hdr)
{
    __shared__ unsigned h[kSortMaxBins];
    __shared__ __align__(16) float spos[FIRST ? 3 * kSortTile : 4];
    const int B = 1 << bits, mask = B - 1;
    for (int d = threadIdx.x; d < B; d += blockDim.x) h[d] = 0u;
    const size_t base = (size_t)blockIdx.x * kSortTile;
    const int n = (int)min((size_t)kSortTile, (size_t)N - base);
    if constexpr (FIRST) stage_positions(pos, base, n, spos);
    __syncthreads();
    bool bad = false;
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
        int key;
        if constexpr (FIRST) {
            float4 r;
            key = particle_key(spos + 3 * l, (int)(base + l), boxes, nboxes, &r, &bad);
        } else {
            key = key_in[base + l];
        }
        atomicAdd(&h[(key >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < B; d += blockDim.x) M[(size_t)d * tiles + blockIdx.x] = h[d];
    if (FIRST && bad) atomicOr(&hdr->status, 1 << NF_ERR_NONFINITE);
}

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

// In-place exclusive scan of a[0 .. n), n <= 2 * blockDim.x, by the whole block.
__device__ __forceinline__ void block_scan_array(unsigned* a, int n)
{
    const int i0 = 2 * threadIdx.x;
    const unsigned v0 = i0 < n ? a[i0] : 0u, v1 = i0 + 1 < n ? a[i0 + 1] : 0u;
    unsigned total;
    const unsigned pre = block_excl_scan(v0 + v1, &total);
    if (i0 < n) a[i0] = pre;
    if (i0 + 1 < n) a[i0 + 1] = pre + v0;
    __syncthreads();
}

// Exclusive scan of uint32 (reduce, scan of block sums, apply)
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

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

// Dynamic shared memory of k_sort_pass for B bins.
__host__ __device__ constexpr size_t sort_smem_bytes(int B)
{
    return (size_t)kSortWarps * B * 4 + (size_t)kSortTile * 16 + (size_t)kSortTile * 4 + 2ull * B * 4;
}

// One stable pass over the digit (key >> shift) & (2^bits - 1).  FIRST reads
// positions and computes keys and offsets; later passes read (rel, key) from
// the previous pass.  LAST also writes perm (the original index) and the keys
// in their final order.
// Resident blocks per SM the register budget is sized for (3: 80 registers;
// measured on GB300 at 512^3: 5.65 ms per binning call against 6.64 ms with 2
// and 5.67 ms with 4).  The pass is bound by latency, so occupancy pays.
// Ranking within a warp: 1 = one ballot per digit bit, 0 = __match_any_sync.
#ifndef NF_SORT_BALLOT
#define NF_SORT_BALLOT 1
#endif
#ifndef NF_SORT_MINB
#define NF_SORT_MINB 3
#endif
template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(kSortWarps * 32, NF_SORT_MINB)
k_sort_pass(const float* __restrict__ pos, const BoxDev* __restrict__ boxes, int nboxes,
            const float4* __restrict__ rel_in, const int* __restrict__ key_in, float4* __restrict__ rel_out,
            int* __restrict__ key_out, int* __restrict__ perm_out, int N, int shift, int bits, int tiles,
            const unsigned* __restrict__ M)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int B = 1 << bits, mask = B - 1;
    unsigned* cnt = reinterpret_cast<unsigned*>(smem);                                // [warps][B]
    float4* sbuf = reinterpret_cast<float4*>(smem + (size_t)kSortWarps * B * 4);      // [tile]
    int* skey = reinterpret_cast<int*>(sbuf + kSortTile);                             // [tile]
    unsigned* s_start = reinterpret_cast<unsigned*>(skey + kSortTile);                // [B] local run starts
    unsigned* s_gbase = s_start + B;                                                  // [B] global run starts

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int tile = blockIdx.x;
    // each warp clears its own row of counts (it alone reads them before the
    // next block-wide barrier)
    unsigned* my = cnt + w * B;
    for (int i = lane; i < B; i += 32) my[i] = 0u;
    __syncwarp();
    for (int d = tid; d < B; d += blockDim.x) s_gbase[d] = M[(size_t)d * tiles + tile];  // scanned: first output slot
    const size_t base = (size_t)tile * kSortTile;
    const int n = (int)min((size_t)kSortTile, (size_t)N - base);
    // the first pass reads the tile's positions into the (still unused) reorder
    // buffer, each warp its own elements
    float* spos = reinterpret_cast<float*>(sbuf);
    if constexpr (FIRST) {
        const int lo = w * 32 * kWarpElems;
        const int nw = n - lo < 0 ? 0 : (n - lo > 32 * kWarpElems ? 32 * kWarpElems : n - lo);
        stage_positions_warp(pos, base + lo, nw, spos + 3 * lo, lane);
    }

    // load: warp w owns the consecutive elements [w*32R, (w+1)*32R) of the tile
    constexpr int R = kSortTile / (kSortWarps * 32);
    float4 v[R];
    int key[R];
    bool bad = false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int l = w * 32 * R + r * 32 + lane;
        key[r] = 0;
        v[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (l < n) {
            const int e = (int)(base + l);
            if constexpr (FIRST) {
                key[r] = particle_key(spos + 3 * l, e, boxes, nboxes, &v[r], &bad);
            } else {
                v[r] = rel_in[e];
                key[r] = key_in[e];
            }
        }
    }
    (void)bad;  // non-finite input is flagged by k_tile_hist

    // stable rank within the tile: by digit, then by position in the tile
    const unsigned lt = (1u << lane) - 1u;
    unsigned rk[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool valid = w * 32 * R + r * 32 + lane < n;
        const int d = valid ? ((key[r] >> shift) & mask) : B;
#if NF_SORT_BALLOT
        // the lanes holding the same digit, one vote per digit bit
        unsigned peers = __ballot_sync(kFull, valid);
        if (!valid) peers = ~peers;
        for (int b = 0; b < bits; ++b) {
            const bool bit = (d >> b) & 1;
            const unsigned bal = __ballot_sync(kFull, bit);
            peers &= bit ? bal : ~bal;
        }
#else
        const unsigned peers = __match_any_sync(kFull, d);
#endif
        const unsigned c = valid ? my[d] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) my[d] = c + __popc(peers);
        __syncwarp();
        rk[r] = c + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: the warps' counts -> exclusive over warps; the tile's total per digit
    for (int d = tid; d < B; d += blockDim.x) {
        unsigned run = 0;
        for (int q = 0; q < kSortWarps; ++q) {
            const unsigned c = cnt[q * B + d];
            cnt[q * B + d] = run;
            run += c;
        }
        s_start[d] = run;
    }
    __syncthreads();
    block_scan_array(s_start, B);  // first slot of every digit's run in the tile
    // output slot of tile position i = s_gbase[d] - s_start[d] + i (mod 2^32; the
    // result is below N): one table read per element below
    for (int d = tid; d < B; d += blockDim.x) s_gbase[d] -= s_start[d];
    // reorder the tile in shared memory
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int l = w * 32 * R + r * 32 + lane;
        if (l < n) {
            const int d = (key[r] >> shift) & mask;
            const unsigned lp = s_start[d] + cnt[w * B + d] + rk[r];
            if (lp < (unsigned)kSortTile) {  // always true when the ranks are consistent
                sbuf[lp] = v[r];
                skey[lp] = key[r];
            }
        }
    }
    __syncthreads();
    // every run goes out contiguously
    for (int i = tid; i < n; i += blockDim.x) {
        const int k = skey[i];
        const int d = (k >> shift) & mask;
        const size_t g = (size_t)(s_gbase[d] + (unsigned)i);
        if (g >= (size_t)N) continue;  // never: the scanned counts keep every run inside the output
        const float4 x = sbuf[i];
        rel_out[g] = x;
        key_out[g] = k;
        if constexpr (LAST) perm_out[g] = __float_as_int(x.w);
    }
}

// cell_offsets[c] = first sorted slot whose key is >= c, for c in [0, C];
// each thread takes four consecutive sorted keys
__global__ void k_cell_off(const int* __restrict__ keys, int N, int C, int* __restrict__ off)
{
    const int nq = (N + 3) >> 2;
    const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const int i0 = 4 * q;
        int k[4];
        if (vec && i0 + 3 < N) {
            const int4 v = reinterpret_cast<const int4*>(keys)[q];
            k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
        } else {
            for (int j = 0; j < 4; ++j) k[j] = i0 + j < N ? keys[i0 + j] : C;
        }
        // ids are in [0, C) by construction; the clamps keep every write inside
        // off[0 .. C] whatever the ids hold
        int prev = i0 > 0 ? min(max(keys[i0 - 1], -1), C - 1) : -1;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            if (i >= N) break;
            const int kj = min(max(k[j], -1), C - 1);
            for (int c = prev + 1; c <= kj; ++c) off[c] = i;
            prev = kj;
            if (i == N - 1)
                for (int c = kj + 1; c <= C; ++c) off[c] = N;
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

SortPlan sort_plan(int64_t N, int64_t C)
{
    SortPlan p{};
    int bits = 1;
    while ((int64_t(1) << bits) < C) ++bits;
    p.passes = (bits + kSortMaxBits - 1) / kSortMaxBits;
    int left = bits, sh = 0;
    for (int k = 0; k < p.passes; ++k) {
        const int b = (left + (p.passes - k) - 1) / (p.passes - k);  // as even as possible
        p.shift[k] = sh;
        p.bits[k] = b;
        sh += b;
        left -= b;
    }
    p.tiles = (int)((N + kSortTile - 1) / kSortTile);
    if (p.tiles < 1) p.tiles = 1;
    return p;
}

size_t sort_matrix_words(const SortPlan& p)
{
    size_t m = 0;
    for (int k = 0; k < p.passes; ++k) m = std::max(m, (size_t)p.tiles << p.bits[k]);
    return m;
}

size_t sort_ctl_bytes(const SortPlan& p)
{
    const size_t m = sort_matrix_words(p);
    return (m + (m + kScanTile - 1) / kScanTile + 64) * 4;  // the count matrix and the scan's block sums
}

cudaError_t run_sort(const SortPlan& p, const float* pos, int N, int C, const BoxDev* boxes, int nboxes,
                     void* ctl, float4* rel_scratch, int* key_a, int* key_b, float4* rel, int* perm, int* cell_off,
                     WsHeader* hdr, cudaStream_t s)
{
    cudaError_t err;
    unsigned* M = static_cast<unsigned*>(ctl);
    unsigned* aux = M + sort_matrix_words(p);
    // buffers: the last pass writes rel and the keys in key_a; the others alternate so
    // that no pass reads the buffer it writes
    const float4* rin = nullptr;
    const int* kin = nullptr;
    for (int k = 0; k < p.passes; ++k) {
        const bool first = k == 0, last = k == p.passes - 1;
        const int from_end = p.passes - 1 - k;  // 0 for the last pass
        float4* rout = (from_end % 2 == 0) ? rel : rel_scratch;
        int* kout = (from_end % 2 == 0) ? key_a : key_b;
        const int B = 1 << p.bits[k];
        const size_t mn = (size_t)p.tiles * B;
        if (first)
            k_tile_hist<true><<<p.tiles, kSortWarps * 32, 0, s>>>(pos, boxes, nboxes, nullptr, N, p.shift[k],
                                                                 p.bits[k], p.tiles, M, hdr);
        else
            k_tile_hist<false><<<p.tiles, kSortWarps * 32, 0, s>>>(pos, boxes, nboxes, kin, N, p.shift[k],
                                                                  p.bits[k], p.tiles, M, hdr);
        count_launches(1);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        const size_t nb = (mn + kScanTile - 1) / kScanTile;
        k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(M, mn, aux);
        k_scan_aux<<<1, kScanThreads, 0, s>>>(aux, nb);
        k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(M, mn, aux);
        count_launches(3);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        const size_t smem = sort_smem_bytes(B);
        typedef void (*PassFn)(const float*, const BoxDev*, int, const float4*, const int*, float4*, int*, int*,
                               int, int, int, int, const unsigned*);
        PassFn fn = first ? (last ? k_sort_pass<true, true> : k_sort_pass<true, false>)
                          : (last ? k_sort_pass<false, true> : k_sort_pass<false, false>);
        if ((err = ensure_smem((const void*)fn, (int)smem, true)) != cudaSuccess) return err;
        fn<<<p.tiles, kSortWarps * 32, smem, s>>>(pos, boxes, nboxes, rin, kin, rout, kout, perm, N, p.shift[k],
                                                  p.bits[k], p.tiles, M);
        count_launches(1);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        rin = rout;
        kin = kout;
    }
    k_cell_off<<<grid_for(((size_t)N + 3) / 4, 256), 256, 0, s>>>(key_a, N, C, cell_off);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nf
