// Near-field force and adjoint on the sorted cell grid.
//
// Work decomposition (pencil on plane).  The paper groups sinks into pencils
// of 2R+1 cells and sources into 2R+1 pencils so that every sink-source cell
// pair is met exactly once and each sink cell collects 2R+1 partial
// accelerations (Sec. "Pencil-on-Pencil").  Here the cell order is z-fastest,
// so the roles are turned to keep every source run contiguous in memory:
//   work item centre (i, j, k):
//     sinks   = cells (i+c, j, k),   c in [-R, R]   (an x-pencil, 2R+1 cells)
//     sources = cells (i, j+b, k+d), b, d in [-R, R] (2R+1 z-runs of 2R+1 cells)
// A sink in cell (x, j, k) meets source cell (x+a, j+b, k+d) in the item
// centred at x+a, with partial slot c = -a + R.  Every (sink, source-cell)
// pair of the (2R+1)^3 stencil is therefore computed exactly once, and each
// sink gets 2R+1 partial sums, one per slot, which k_combine adds without
// rounding error (an FP32 TwoSum cascade into a hi/lo pair).
// Coordinates are cell-relative FP32 offsets shifted into the frame of the
// item's centre cell (the paper's pencil-centred coordinates, Sec.
// "Pencil-on-Pencil"), so the periodic wrap costs nothing in the pair loop.
//
// Scheduling.  A pencil's sinks are cut into chunks of 32 * SMAX; one chunk
// is one work item for one warp.  k_pencils/k_items build the item list in
// descending cost order (cost buckets of half powers of two: longest first,
// as the paper's NUMA scheduler hands out work from a shared counter, Sec.
// "Memory and Threads"), and the persistent kernel's warps pull items from an
// atomic counter until the list is exhausted.
//
// Pair loop (one warp, one item).  Each lane keeps S <= SMAX sinks in
// registers (S = ceil(chunk size / 32) is picked per item).  Sources are
// staged B at a time into the warp's shared-memory buffers (double-buffered:
// the next stage's global loads are issued before the current stage is
// computed), shifted into the item's frame as they are staged.  Every lane
// then reads each source with a broadcast shared load and accumulates S pairs
// in FP32 with MUFU rsqrt.  Sums are kept per stage and added into the
// running total after each stage (per-stage partial sums bound the FP32
// accumulation error).
//
// Spline hand-off.  Eq. (spline) switches to 1/r^3 at r = eps_s.  The paper's
// kernel takes min(poly, r^-3) instead of a branch (Sec. "Force Kernel");
// that identity holds because u^3 poly(u) - 1 = -(1-u)^3 (6u^2+3u+1).  Here
// the min form is the exact path ("slow").  A stage whose sources are all
// farther than eps_s from every sink gives the same value with f = r^-3
// alone, so the "fast" path computes only that and tracks the smallest r^2
// it met; if any lane saw r < eps_s, the warp recomputes the stage with the
// exact path.  The source list puts the item's centre cell first, in stages
// of its own; the other source cells follow in rings around it (c_ring).
// A chunk with sinks in the centre cell meets its self pairs there and runs
// those stages on the exact path from the start; any other chunk runs them
// on the tracked fast path like the rest of the first ring.
#include <cuda_runtime.h>

#include "nf_internal.cuh"

namespace nf {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kTiny = 1e-25f;     // r^2 floor: coincident pairs stay finite (r^-3 < FLT_MAX)
constexpr float kFarSrc = 1e18f;    // padding source coordinate: adds exactly 0
constexpr float kFarSink = -1e18f;  // padding sink coordinate
constexpr float kBig = 3.0e38f;

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int wrap(int a, int K)
{
    a %= K;
    return a < 0 ? a + K : a;
}

__device__ __forceinline__ int find_box_by_cell(const BoxDev* boxes, int nboxes, int g)
{
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].cell_base <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}


// Source cells of an item, (b, d) offsets in the plane, in rings around the
// centre: the centre, its 8 neighbours, then rings 2, 3, 4 (the first
// (2R+1)^2 entries are exactly the cells of the stencil for any R <= 4).
// A ball of radius at most one cell around a sink of the pencil reaches only
// the centre and its first ring, so the density estimate needs only those.
__constant__ signed char c_ring[81][2] = {
    {0, 0}, {-1, -1}, {-1, 0}, {-1, 1}, {0, -1}, {0, 1}, {1, -1}, {1, 0}, {1, 1}, {-2, -2}, {-2, -1}, {-2, 0},
    {-2, 1}, {-2, 2}, {-1, -2}, {-1, 2}, {0, -2}, {0, 2}, {1, -2}, {1, 2}, {2, -2}, {2, -1}, {2, 0}, {2, 1},
    {2, 2}, {-3, -3}, {-3, -2}, {-3, -1}, {-3, 0}, {-3, 1}, {-3, 2}, {-3, 3}, {-2, -3}, {-2, 3}, {-1, -3}, {-1, 3},
    {0, -3}, {0, 3}, {1, -3}, {1, 3}, {2, -3}, {2, 3}, {3, -3}, {3, -2}, {3, -1}, {3, 0}, {3, 1}, {3, 2},
    {3, 3}, {-4, -4}, {-4, -3}, {-4, -2}, {-4, -1}, {-4, 0}, {-4, 1}, {-4, 2}, {-4, 3}, {-4, 4}, {-3, -4}, {-3, 4},
    {-2, -4}, {-2, 4}, {-1, -4}, {-1, 4}, {0, -4}, {0, 4}, {1, -4}, {1, 4}, {2, -4}, {2, 4}, {3, -4}, {3, 4},
    {4, -4}, {4, -3}, {4, -2}, {4, -1}, {4, 0}, {4, 1}, {4, 2}, {4, 3}, {4, 4}};
static_assert(NF_MAX_R <= 4, "the ring table covers R <= 4");

__device__ __forceinline__ int cell_count(const int* off, int cid, int* start)
{
    int s = off[cid];
    *start = s;
    return off[cid + 1] - s;
}

__device__ __forceinline__ int cost_bucket(unsigned long long cost)
{
    if (cost == 0) return kBuckets - 1;
    int h = (int)floorf(2.0f * log2f((float)cost));
    int b = (kBuckets - 2) - h;
    return b < 0 ? 0 : (b > kBuckets - 2 ? kBuckets - 2 : b);
}

// ---------------------------------------------------------------------------
// Work list
// ---------------------------------------------------------------------------

__global__ void k_pencils(const BoxDev* __restrict__ boxes, int nboxes, int Ctot,
                          const int* __restrict__ off, int CH, int SB, int* __restrict__ chunks,
                          unsigned* __restrict__ bucket_count, unsigned char* __restrict__ bucket_of,
                          WsHeader* hdr)
{
    unsigned long long pairs = 0, lane_pairs = 0, stages = 0, stages_exact = 0;
    int max_occ = 0;
    // every lane of a warp runs the same iterations (blockDim is a multiple of
    // 32), so the warp-wide votes below see all 32 lanes
    for (int gb = blockIdx.x * blockDim.x; gb < Ctot; gb += gridDim.x * blockDim.x) {
        const int g = gb + (int)threadIdx.x;
        int nch = 0, bk = 0;
        if (g < Ctot) {
            const BoxDev& B = boxes[find_box_by_cell(boxes, nboxes, g)];
            const int K = B.K, R = B.R, cb = B.cell_base;
            const int l = g - cb;
            const int i = l / (K * K), j = (l / K) % K, k = l % K;
            int st;
            int n_sink = 0, c_first = 0;
            for (int c = -R; c <= R; ++c) {
                if (c == 0) c_first = n_sink;
                n_sink += cell_count(off, cb + (wrap(i + c, K) * K + j) * K + k, &st);
            }
            int n_src = 0;
            for (int b = -R; b <= R; ++b)
                for (int d = -R; d <= R; ++d)
                    n_src += cell_count(off, cb + (i * K + wrap(j + b, K)) * K + wrap(k + d, K), &st);
            int occ = cell_count(off, g, &st);
            max_occ = max(max_occ, occ);
            nch = (n_sink + CH - 1) / CH;
            chunks[g] = nch;
            unsigned long long cost = (unsigned long long)n_src * (unsigned long long)min(n_sink, CH);
            bk = cost_bucket(cost);
            bucket_of[g] = (unsigned char)bk;
            pairs += (unsigned long long)n_sink * (unsigned long long)n_src;
            // every chunk of this pencil runs the centre cell's sources in stages of their
            // own and the rest in stages of SB (the pair kernel's stage_range); the
            // chunks holding sinks of the centre cell run those stages exactly
            const int st0 = (occ + SB - 1) / SB;
            stages += (unsigned long long)nch * (unsigned long long)(st0 + (n_src - occ + SB - 1) / SB);
            if (occ > 0) {
                const int self_chunks = (c_first + occ + CH - 1) / CH - c_first / CH;
                stages_exact += (unsigned long long)self_chunks * (unsigned long long)st0;
            }
            if (nch) {
                int rem = n_sink - (nch - 1) * CH;
                unsigned long long lanes = (unsigned long long)(nch - 1) * CH + 32ull * ((rem + 31) / 32);
                lane_pairs += lanes * (unsigned long long)n_src;
            }
        }
        // one atomic per bucket per warp: most cells of a box fall in a few buckets
        const int key = nch ? bk : -1;
        const unsigned peers = __match_any_sync(kFull, key);
        const unsigned tot = __reduce_add_sync(peers, (unsigned)nch);
        if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&bucket_count[bk], tot);
    }
    for (int o = 16; o; o >>= 1) {
        pairs += __shfl_xor_sync(kFull, pairs, o);
        lane_pairs += __shfl_xor_sync(kFull, lane_pairs, o);
        stages += __shfl_xor_sync(kFull, stages, o);
        stages_exact += __shfl_xor_sync(kFull, stages_exact, o);
        max_occ = max(max_occ, __shfl_xor_sync(kFull, max_occ, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&hdr->pairs, pairs);
        atomicAdd(&hdr->lane_pairs, lane_pairs);
        atomicAdd(&hdr->stages, stages);
        atomicAdd(&hdr->stages_exact, stages_exact);
        atomicMax(&hdr->max_occ, max_occ);
    }
}

// Exclusive scan of the bucket counts (one warp pair of lanes per bucket);
// writes the total to the header.
__global__ void k_bucket_scan(unsigned* bucket_count, WsHeader* hdr)
{
    __shared__ unsigned v[kBuckets];
    int t = threadIdx.x;
    v[t] = bucket_count[t];
    __syncthreads();
    if (t == 0) {
        unsigned run = 0;
        for (int b = 0; b < kBuckets; ++b) {
            unsigned c = v[b];
            v[b] = run;
            run += c;
        }
        hdr->n_items = (int)run;
    }
    __syncthreads();
    bucket_count[t] = v[t];
}

__global__ void k_items(const BoxDev* __restrict__ boxes, int nboxes, int Ctot,
                        const int* __restrict__ chunks, const unsigned char* __restrict__ bucket_of,
                        unsigned* __restrict__ cursor, int4* __restrict__ items)
{
    // every lane of a warp runs the same iterations (blockDim is a multiple of 32)
    const int lane = threadIdx.x & 31;
    for (int gb = blockIdx.x * blockDim.x; gb < Ctot; gb += gridDim.x * blockDim.x) {
        const int g = gb + (int)threadIdx.x;
        const int nch = g < Ctot ? chunks[g] : 0;
        const int bk = nch ? (int)bucket_of[g] : -1;
        // one atomic per bucket per warp; each lane's chunks follow those of the
        // lanes below it in the same bucket (the order of items within a bucket
        // does not change any result)
        const unsigned peers = __match_any_sync(kFull, bk);
        const int leader = __ffs(peers) - 1;
        unsigned pre = 0, tot = 0;
        for (int src = 0; src < 32; ++src) {
            const unsigned v = __shfl_sync(kFull, (unsigned)nch, src);
            if ((peers >> src) & 1u) {
                tot += v;
                if (src < lane) pre += v;
            }
        }
        unsigned base = 0;
        if (nch && lane == leader) base = atomicAdd(&cursor[bk], tot);
        base = __shfl_sync(kFull, base, leader) + pre;
        if (nch) {
            const int b = find_box_by_cell(boxes, nboxes, g);
            for (int q = 0; q < nch; ++q) items[base + q] = make_int4(g, q, b, 0);
        }
    }
}

__global__ void k_gather_g(const float* __restrict__ g, const int* __restrict__ perm, int Ntot,
                           float4* __restrict__ gs)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < Ntot; s += gridDim.x * blockDim.x) {
        int e = perm[s];
        gs[s] = make_float4(g[3 * (size_t)e + 0], g[3 * (size_t)e + 1], g[3 * (size_t)e + 2], 0.0f);
    }
}

// ---------------------------------------------------------------------------
// Pair arithmetic
// ---------------------------------------------------------------------------

struct Coef {
    float c0, c1, c2;  // Eq. (spline) polynomial in cell units: c0 + r^2 (c2 + c1/r)
    float e0, e1;      // f'(r)/r inside the softening: e1 + e0/r
    float eps2;
    int dens_defer;    // top hat only in stages where some lane met r < b
};

// Packed FP32x2 arithmetic (sm_100+ `add/mul/fma.rn.f32x2`): one instruction
// works on the two halves of a 64-bit register pair.  The pair loops put two
// sources side by side in each pair, so every instruction computes two
// interactions of one sink; this halves the issue slots of the FP32 work.
typedef unsigned long long f2;

// Where r^-2 comes from in the fast paths: 1 = MUFU reciprocal, 0 = r^-1 * r^-1
// on the FMA pipe.  Measured on GB300: the MUFU unit (16 lanes per clock per
// SM) is already the second bottleneck beside the FMA pipe with one rsqrt per
// pair, so both directions take r^-2 from the FMA pipe.
#ifndef NF_FWD_RCP
#define NF_FWD_RCP 0
#endif
#ifndef NF_ADJ_RCP
#define NF_ADJ_RCP 0
#endif
// Unroll depth of the fast pair loops over groups of four sources, with the
// r^2 tracking (stages near the sink) and without it (_FAR: the stages of
// ring 2 and beyond, which need fewer registers).  Measured on GB300: any
// unrolling is slower inside the kernel (forward, four sinks per lane, 256^3
// clustered: 78.8 ms, 83.1 ms unrolled by two, 89.1 ms by four), although the
// loop body alone gains from it.
#ifndef NF_FWD_UNROLL
#define NF_FWD_UNROLL 1
#endif
#ifndef NF_ADJ_UNROLL
#define NF_ADJ_UNROLL 1
#endif
#ifndef NF_FWD_UNROLL_FAR
#define NF_FWD_UNROLL_FAR 1
#endif
#ifndef NF_ADJ_UNROLL_FAR
#define NF_ADJ_UNROLL_FAR 1
#endif
constexpr int kFwdUnroll = NF_FWD_UNROLL;
constexpr int kAdjUnroll = NF_ADJ_UNROLL;
constexpr int kFwdUnrollFar = NF_FWD_UNROLL_FAR;
constexpr int kAdjUnrollFar = NF_ADJ_UNROLL_FAR;

__device__ __forceinline__ f2 pk(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
// one half of a packed pair (the unpack names both halves; one is unused)
#pragma nv_diag_suppress 550
__device__ __forceinline__ float lo(f2 v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}
__device__ __forceinline__ float hi(f2 v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}
#pragma nv_diag_default 550
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ f2 rsqrt2(f2 v) { return pk(rsqrt_approx(lo(v)), rsqrt_approx(hi(v))); }
// Smallest r^2 met so far, updated with both halves of a packed r^2: one
// three-input min (sm_100 and later) instead of two.
#ifndef NF_MIN3
#define NF_MIN3 1
#endif
__device__ __forceinline__ float track_min(float t, f2 r2)
{
#if NF_MIN3
    float m;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(t), "f"(lo(r2)), "f"(hi(r2)));
    return m;
#else
    return fminf(t, fminf(lo(r2), hi(r2)));
#endif
}
// r^-2 from the MUFU reciprocal: keeps the FMA pipe (the bottleneck) for the sums
__device__ __forceinline__ f2 rcp2(f2 v) { return pk(rcp_approx(lo(v)), rcp_approx(hi(v))); }

// Per-lane sink state.  Positions and gradients are held negated and
// duplicated in both halves ({-x, -x}), so d = source + sink is one add2.
template <int S>
struct SinkSet {
    f2 nx[S], ny[S], nz[S];   // -position
    f2 ngx[S], ngy[S], ngz[S];  // -g (adjoint)
    f2 sx[S], sy[S], sz[S];   // current stage, even/odd sources in the halves
    f2 sw[S];                 // current stage, density estimate
    float ax[S], ay[S], az[S];  // running totals
    float aw[S];              // running density estimate
};

// Stage buffers of one warp in shared memory: sources as structure of arrays,
// four consecutive sources per 16-byte word.
struct StageView {
    const float4* X;
    const float4* Y;
    const float4* Z;
    const float4* GX;
    const float4* GY;
    const float4* GZ;
};

// Top-hat density term of one packed pair (Sec. "Force Kernel"): b^2 - r^2 where positive.
__device__ __forceinline__ f2 tophat2(f2 r2, f2 b2)
{
    const f2 t = fma2(r2, pk(-1.0f, -1.0f), b2);
    return pk(fmaxf(lo(t), 0.0f), fmaxf(hi(t), 0.0f));
}

// Forward, fast path: f = r^-3 for every pair; TRK tracks the smallest r^2.
// DENS adds the top-hat density estimate as a 4th sum.
template <int S, bool DENS, bool TRK = true>
__device__ __forceinline__ void stage_fwd_fast(const StageView& v, int cnt, SinkSet<S>& k, float& trk, f2 b2)
{
    const f2 tiny = pk(kTiny, kTiny);
#pragma unroll (TRK ? kFwdUnroll : kFwdUnrollFar)
    for (int q = 0; q < cnt; q += 4) {
        const float4 xs = v.X[q >> 2], ys = v.Y[q >> 2], zs = v.Z[q >> 2];
        const f2 px[2] = {pk(xs.x, xs.y), pk(xs.z, xs.w)};
        const f2 py[2] = {pk(ys.x, ys.y), pk(ys.z, ys.w)};
        const f2 pz[2] = {pk(zs.x, zs.y), pk(zs.z, zs.w)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const f2 dx = add2(px[h], k.nx[s]), dy = add2(py[h], k.ny[s]), dz = add2(pz[h], k.nz[s]);
                f2 r2 = fma2(dx, dx, tiny);
                r2 = fma2(dy, dy, r2);
                r2 = fma2(dz, dz, r2);
                if constexpr (TRK) trk = track_min(trk, r2);
                if constexpr (DENS) k.sw[s] = add2(k.sw[s], tophat2(r2, b2));
#if NF_FWD_RCP
                const f2 f = mul2(rcp2(r2), rsqrt2(r2));
#else
                const f2 ri = rsqrt2(r2);
                const f2 f = mul2(mul2(ri, ri), ri);
#endif
                k.sx[s] = fma2(dx, f, k.sx[s]);
                k.sy[s] = fma2(dy, f, k.sy[s]);
                k.sz[s] = fma2(dz, f, k.sz[s]);
            }
        }
    }
}

// Top-hat density term alone, for a stage in which some pair is closer than b
// (the deferred mode): the same operations in the same order as the fused
// term of stage_fwd_fast, so both modes give bit-identical sums.
template <int S>
__device__ __forceinline__ void stage_density(const StageView& v, int cnt, SinkSet<S>& k, f2 b2)
{
    const f2 tiny = pk(kTiny, kTiny);
#pragma unroll 1
    for (int q = 0; q < cnt; q += 4) {
        const float4 xs = v.X[q >> 2], ys = v.Y[q >> 2], zs = v.Z[q >> 2];
        const f2 px[2] = {pk(xs.x, xs.y), pk(xs.z, xs.w)};
        const f2 py[2] = {pk(ys.x, ys.y), pk(ys.z, ys.w)};
        const f2 pz[2] = {pk(zs.x, zs.y), pk(zs.z, zs.w)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const f2 dx = add2(px[h], k.nx[s]), dy = add2(py[h], k.ny[s]), dz = add2(pz[h], k.nz[s]);
                f2 r2 = fma2(dx, dx, tiny);
                r2 = fma2(dy, dy, r2);
                r2 = fma2(dz, dz, r2);
                k.sw[s] = add2(k.sw[s], tophat2(r2, b2));
            }
        }
    }
}

// Forward, exact path: f = min(poly(r), r^-3) (Eq. (spline) with the min hand-off).
template <int S, bool DENS>
__device__ __forceinline__ void stage_fwd_exact(const StageView& v, int cnt, SinkSet<S>& k, const Coef& cf, f2 b2)
{
    const f2 tiny = pk(kTiny, kTiny);
    const f2 c0 = pk(cf.c0, cf.c0), c1 = pk(cf.c1, cf.c1), c2 = pk(cf.c2, cf.c2);
#pragma unroll 1
    for (int q = 0; q < cnt; q += 4) {
        const float4 xs = v.X[q >> 2], ys = v.Y[q >> 2], zs = v.Z[q >> 2];
        const f2 px[2] = {pk(xs.x, xs.y), pk(xs.z, xs.w)};
        const f2 py[2] = {pk(ys.x, ys.y), pk(ys.z, ys.w)};
        const f2 pz[2] = {pk(zs.x, zs.y), pk(zs.z, zs.w)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const f2 dx = add2(px[h], k.nx[s]), dy = add2(py[h], k.ny[s]), dz = add2(pz[h], k.nz[s]);
                f2 r2 = fma2(dx, dx, tiny);
                r2 = fma2(dy, dy, r2);
                r2 = fma2(dz, dz, r2);
                if constexpr (DENS) k.sw[s] = add2(k.sw[s], tophat2(r2, b2));
                const f2 ri = rsqrt2(r2);
                const f2 p = fma2(r2, fma2(c1, ri, c2), c0);
                const f2 r3 = mul2(mul2(ri, ri), ri);
                const f2 f = pk(fminf(lo(p), lo(r3)), fminf(hi(p), hi(r3)));
                k.sx[s] = fma2(dx, f, k.sx[s]);
                k.sy[s] = fma2(dy, f, k.sy[s]);
                k.sz[s] = fma2(dz, f, k.sz[s]);
            }
        }
    }
}

// Adjoint, fast path: J v = r^-3 (v - 3 r^-2 (d.v) d), v = g_j - g_i; TRK
// tracks the smallest r^2.
template <int S, bool TRK = true>
__device__ __forceinline__ void stage_adj_fast(const StageView& v, int cnt, SinkSet<S>& k, float& trk)
{
    const f2 tiny = pk(kTiny, kTiny);
    const f2 m3 = pk(-3.0f, -3.0f);
#pragma unroll (TRK ? kAdjUnroll : kAdjUnrollFar)
    for (int q = 0; q < cnt; q += 4) {
        const float4 xs = v.X[q >> 2], ys = v.Y[q >> 2], zs = v.Z[q >> 2];
        const float4 gxs = v.GX[q >> 2], gys = v.GY[q >> 2], gzs = v.GZ[q >> 2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const f2 px = h ? pk(xs.z, xs.w) : pk(xs.x, xs.y);
            const f2 py = h ? pk(ys.z, ys.w) : pk(ys.x, ys.y);
            const f2 pz = h ? pk(zs.z, zs.w) : pk(zs.x, zs.y);
            const f2 qx = h ? pk(gxs.z, gxs.w) : pk(gxs.x, gxs.y);
            const f2 qy = h ? pk(gys.z, gys.w) : pk(gys.x, gys.y);
            const f2 qz = h ? pk(gzs.z, gzs.w) : pk(gzs.x, gzs.y);
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const f2 dx = add2(px, k.nx[s]), dy = add2(py, k.ny[s]), dz = add2(pz, k.nz[s]);
                f2 r2 = fma2(dx, dx, tiny);
                r2 = fma2(dy, dy, r2);
                r2 = fma2(dz, dz, r2);
                if constexpr (TRK) trk = track_min(trk, r2);
#if NF_ADJ_RCP
                const f2 ri2 = rcp2(r2);
                const f2 ri3 = mul2(ri2, rsqrt2(r2));
#else
                const f2 ri = rsqrt2(r2);
                const f2 ri2 = mul2(ri, ri);
                const f2 ri3 = mul2(ri2, ri);
#endif
                const f2 vx = add2(qx, k.ngx[s]), vy = add2(qy, k.ngy[s]), vz = add2(qz, k.ngz[s]);
                f2 dv = mul2(dx, vx);
                dv = fma2(dy, vy, dv);
                dv = fma2(dz, vz, dv);
                const f2 c = mul2(dv, mul2(ri2, m3));
                k.sx[s] = fma2(ri3, fma2(c, dx, vx), k.sx[s]);
                k.sy[s] = fma2(ri3, fma2(c, dy, vy), k.sy[s]);
                k.sz[s] = fma2(ri3, fma2(c, dz, vz), k.sz[s]);
            }
        }
    }
}

// Adjoint, exact path: J v = F (v + G (d.v) d), F = f and G = (f'/r) / f,
// with the softened branch of Eq. (spline) selected per pair for r^2 < eps_s^2
// (F = poly/eps_s^3, f'/r = e1 + e0/r; outside F = r^-3, G = -3 r^-2).
template <int S>
__device__ __forceinline__ void stage_adj_exact(const StageView& v, int cnt, SinkSet<S>& k, const Coef& cf)
{
    const f2 tiny = pk(kTiny, kTiny);
    const f2 m3 = pk(-3.0f, -3.0f);
    const f2 c0 = pk(cf.c0, cf.c0), c1 = pk(cf.c1, cf.c1), c2 = pk(cf.c2, cf.c2);
    const f2 e0 = pk(cf.e0, cf.e0), e1 = pk(cf.e1, cf.e1);
#pragma unroll 1
    for (int q = 0; q < cnt; q += 4) {
        const float4 xs = v.X[q >> 2], ys = v.Y[q >> 2], zs = v.Z[q >> 2];
        const float4 gxs = v.GX[q >> 2], gys = v.GY[q >> 2], gzs = v.GZ[q >> 2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const f2 px = h ? pk(xs.z, xs.w) : pk(xs.x, xs.y);
            const f2 py = h ? pk(ys.z, ys.w) : pk(ys.x, ys.y);
            const f2 pz = h ? pk(zs.z, zs.w) : pk(zs.x, zs.y);
            const f2 qx = h ? pk(gxs.z, gxs.w) : pk(gxs.x, gxs.y);
            const f2 qy = h ? pk(gys.z, gys.w) : pk(gys.x, gys.y);
            const f2 qz = h ? pk(gzs.z, gzs.w) : pk(gzs.x, gzs.y);
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const f2 dx = add2(px, k.nx[s]), dy = add2(py, k.ny[s]), dz = add2(pz, k.nz[s]);
                f2 r2 = fma2(dx, dx, tiny);
                r2 = fma2(dy, dy, r2);
                r2 = fma2(dz, dz, r2);
                const f2 ri = rsqrt2(r2);
                const f2 ri2 = rcp2(r2);
                const f2 Fs = fma2(r2, fma2(c1, ri, c2), c0);
                const f2 Gs = mul2(fma2(e0, ri, e1), rcp2(Fs));
                const f2 Fr = mul2(ri2, ri);
                const f2 Gr = mul2(ri2, m3);
                const bool sl = lo(r2) < cf.eps2, sh = hi(r2) < cf.eps2;
                const f2 F = pk(sl ? lo(Fs) : lo(Fr), sh ? hi(Fs) : hi(Fr));
                const f2 G = pk(sl ? lo(Gs) : lo(Gr), sh ? hi(Gs) : hi(Gr));
                const f2 vx = add2(qx, k.ngx[s]), vy = add2(qy, k.ngy[s]), vz = add2(qz, k.ngz[s]);
                f2 dv = mul2(dx, vx);
                dv = fma2(dy, vy, dv);
                dv = fma2(dz, vz, dv);
                const f2 c = mul2(dv, G);
                k.sx[s] = fma2(F, fma2(c, dx, vx), k.sx[s]);
                k.sy[s] = fma2(F, fma2(c, dy, vy), k.sy[s]);
                k.sz[s] = fma2(F, fma2(c, dz, vz), k.sz[s]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Persistent kernel
// ---------------------------------------------------------------------------

template <int B, bool ADJ>
struct WarpSmem {
    // raw[2][B] float4 and graw[2][B] float4 (adjoint): cp.async targets;
    // soa[3 or 6][B] floats: X, Y, Z (and GX, GY, GZ) of the stage being
    // computed (written by the fix-up pass after the previous stage finished);
    // sh[2][B] float2: (dy, dz) frame shift of each staged source;
    // then the segment table: seg_pre[max_nseg + 1], seg_start, seg_dy, seg_dz.
    static constexpr int NC = ADJ ? 6 : 3;
    static constexpr size_t raw_bytes = 2ull * B * sizeof(float4);
    static constexpr size_t graw_bytes = ADJ ? 2ull * B * sizeof(float4) : 0;
    static constexpr size_t soa_bytes = 1ull * NC * B * sizeof(float);
    static constexpr size_t sh_bytes = 2ull * B * sizeof(float2);
    static size_t __host__ __device__ bytes(int max_nseg)
    {
        size_t t = (size_t)(4 * max_nseg + 1) * 4;
        return raw_bytes + graw_bytes + soa_bytes + sh_bytes + ((t + 15) & ~size_t(15));
    }
};

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

struct ItemCtx {
    int K, R, cb;
    int i, j, k;
    int ns;           // 2R+1
    int sc_start;     // lane c < ns: first sorted slot of sink cell c
    int sc_cnt;       // lane c < ns: occupancy of sink cell c
    int sc_incl;      // lane c < ns: inclusive prefix of sink counts
    int n_sink;
    int chunk_begin;
    int n_src;
    int n_c0;         // sources of the centre cell (processed first, exact path)
    int n_near;       // sources of the centre cell and its first ring
    bool has_self;    // some sink of this chunk lies in the centre cell (self pairs)
    bool near_x;      // some sink of this chunk lies within one cell (in x) of the source plane
};

// Sorted slot and partial slot of the sink at pencil position p.
__device__ __forceinline__ void sink_lookup(const ItemCtx& it, int p, int* at, int* slot)
{
    int c_sel = 0, a = 0;
    for (int c = 0; c < it.ns; ++c) {
        int inc = __shfl_sync(kFull, it.sc_incl, c);
        int cnt = __shfl_sync(kFull, it.sc_cnt, c);
        int st = __shfl_sync(kFull, it.sc_start, c);
        if (p >= inc - cnt && p < inc) {
            c_sel = c;
            a = st + (p - (inc - cnt));
        }
    }
    *at = a;
    *slot = c_sel;
}

struct WarpBufs {
    float4* raw;    // [2][B]
    float4* graw;   // [2][B] (adjoint)
    float* soa;     // [NC][B]
    float2* sh;     // [2][B]
};

template <int S, int B, bool ADJ, bool DENS>
__device__ __forceinline__ void run_item(const ItemCtx& it, const Coef& cf, f2 b2,
                                         const float4* __restrict__ rel, const float4* __restrict__ gs,
                                         const WarpBufs& wb, const int* seg_pre,
                                         const int* seg_start, const float* seg_dy, const float* seg_dz,
                                         float4* __restrict__ partial, int pstride, WsHeader* hdr)
{
    const int lane = threadIdx.x & 31;
    SinkSet<S> k;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int p = it.chunk_begin + s * 32 + lane;
        int at, slot;
        sink_lookup(it, p, &at, &slot);
        const bool ok = p < it.n_sink;
        float4 r = ok ? rel[at] : make_float4(kFarSink, kFarSink, kFarSink, 0.0f);
        const float x = r.x + (float)(slot - it.R);
        k.nx[s] = pk(-x, -x);
        k.ny[s] = pk(-r.y, -r.y);
        k.nz[s] = pk(-r.z, -r.z);
        if constexpr (ADJ) {
            float4 g = ok ? gs[at] : make_float4(0.f, 0.f, 0.f, 0.f);
            k.ngx[s] = pk(-g.x, -g.x);
            k.ngy[s] = pk(-g.y, -g.y);
            k.ngz[s] = pk(-g.z, -g.z);
        }
        k.ax[s] = k.ay[s] = k.az[s] = 0.0f;
        k.aw[s] = 0.0f;
    }

    constexpr int PER = B / 32;
    const bool dens_near_only = lo(b2) <= 1.0f;    // b <= one cell width
    const bool soft_near_only = cf.eps2 <= 1.0f;   // eps_s <= one cell width
    // deferred top hat (small b): the fast path tracks the smallest r^2 of the
    // stage anyway, and the term is added only where it is below b^2
    const bool dens_defer = DENS && cf.dens_defer != 0 && dens_near_only;
    const int nst0 = (it.n_c0 + B - 1) / B;
    const int nst = nst0 + (it.n_src - it.n_c0 + B - 1) / B;
    int cur = 0;

    auto stage_range = [&](int st, int& beg, int& end) {
        if (st < nst0) {
            beg = st * B;
            end = min(beg + B, it.n_c0);
        } else {
            beg = it.n_c0 + (st - nst0) * B;
            end = min(beg + B, it.n_src);
        }
    };
    // Issue the asynchronous copies of stage st into buffer buf.  Each lane
    // copies the sources it will later shift and transpose.
    auto issue = [&](int st, int buf) {
        int beg, end;
        stage_range(st, beg, end);
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int p = beg + t * 32 + lane;
            const int slot = buf * B + t * 32 + lane;
            if (p < end) {
                while (p >= seg_pre[cur + 1]) ++cur;
                const int at = seg_start[cur] + (p - seg_pre[cur]);
                cp_async16(&wb.raw[slot], &rel[at]);
                if constexpr (ADJ) cp_async16(&wb.graw[slot], &gs[at]);
                wb.sh[slot] = make_float2(seg_dy[cur], seg_dz[cur]);
            } else {
                wb.raw[slot] = make_float4(kFarSrc, kFarSrc, kFarSrc, 0.0f);
                if constexpr (ADJ) wb.graw[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
                wb.sh[slot] = make_float2(0.0f, 0.0f);
            }
        }
        cp_async_commit();
    };
    // Shift this lane's own staged sources into the item's frame and write
    // them to the structure-of-arrays buffers the pair loop reads.
    auto fixup = [&](int buf) {
        float* soa = wb.soa;
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int i = t * 32 + lane;
            const float4 v = wb.raw[buf * B + i];
            const float2 sh = wb.sh[buf * B + i];
            soa[0 * B + i] = v.x;
            soa[1 * B + i] = v.y + sh.x;
            soa[2 * B + i] = v.z + sh.y;
            if constexpr (ADJ) {
                const float4 g = wb.graw[buf * B + i];
                soa[3 * B + i] = g.x;
                soa[4 * B + i] = g.y;
                soa[5 * B + i] = g.z;
            }
        }
    };

    if (nst > 0) issue(0, 0);
    for (int st = 0; st < nst; ++st) {
        const int buf = st & 1;
        if (st + 1 < nst) {
            issue(st + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        fixup(buf);
        __syncwarp();
        int beg, end;
        stage_range(st, beg, end);
        const int cnt = (end - beg + 7) & ~7;
        const float* soa = wb.soa;
        StageView v;
        v.X = reinterpret_cast<const float4*>(soa + 0 * B);
        v.Y = reinterpret_cast<const float4*>(soa + 1 * B);
        v.Z = reinterpret_cast<const float4*>(soa + 2 * B);
        v.GX = reinterpret_cast<const float4*>(soa + (ADJ ? 3 : 0) * B);
        v.GY = reinterpret_cast<const float4*>(soa + (ADJ ? 4 : 0) * B);
        v.GZ = reinterpret_cast<const float4*>(soa + (ADJ ? 5 : 0) * B);
        // the centre cell's stages hold the self pairs only for chunks with sinks
        // in that cell; other chunks run them on the tracked fast path
        bool exact = it.has_self && st < nst0;
        // Sources of ring 2 and beyond are at least one cell away from every
        // sink of the pencil, and every source is more than one cell away from
        // the sinks of cells two or more cells from the plane in x: the top hat
        // (b <= one cell) and the softened branch (eps_s <= one cell) cannot
        // occur there.
        const bool far = beg >= it.n_near || !it.near_x;
        const bool dens = DENS && (!dens_near_only || !far);
        if (!exact) {
#pragma unroll
            for (int s = 0; s < S; ++s) k.sx[s] = k.sy[s] = k.sz[s] = k.sw[s] = 0ull;
            float trk = kBig;
            if (far && soft_near_only) {
                if constexpr (ADJ) stage_adj_fast<S, false>(v, cnt, k, trk);
                else if (dens) stage_fwd_fast<S, DENS, false>(v, cnt, k, trk, b2);
                else stage_fwd_fast<S, false, false>(v, cnt, k, trk, b2);
            } else {
                if constexpr (ADJ) stage_adj_fast<S>(v, cnt, k, trk);
                else if (dens && !dens_defer) stage_fwd_fast<S, DENS>(v, cnt, k, trk, b2);
                else stage_fwd_fast<S, false>(v, cnt, k, trk, b2);
                exact = __any_sync(kFull, trk < cf.eps2);
                if (exact && lane == 0) atomicAdd(&hdr->stages_rerun, 1ull);  // rare
                if constexpr (DENS && !ADJ) {
                    // a pair closer than b gives a positive term; elsewhere every term is +0
                    if (dens && dens_defer && !exact && __any_sync(kFull, trk < lo(b2)))
                        stage_density<S>(v, cnt, k, b2);
                }
            }
        }
        if (exact) {
#pragma unroll
            for (int s = 0; s < S; ++s) k.sx[s] = k.sy[s] = k.sz[s] = k.sw[s] = 0ull;
            if constexpr (ADJ) stage_adj_exact<S>(v, cnt, k, cf);
            else if (dens) stage_fwd_exact<S, DENS>(v, cnt, k, cf, b2);
            else stage_fwd_exact<S, false>(v, cnt, k, cf, b2);
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            k.ax[s] += lo(k.sx[s]) + hi(k.sx[s]);
            k.ay[s] += lo(k.sy[s]) + hi(k.sy[s]);
            k.az[s] += lo(k.sz[s]) + hi(k.sz[s]);
            if constexpr (DENS) k.aw[s] += lo(k.sw[s]) + hi(k.sw[s]);
        }
        __syncwarp();
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int p = it.chunk_begin + s * 32 + lane;
        int at, slot;
        sink_lookup(it, p, &at, &slot);
        if (p < it.n_sink) {
            // the sink's row of partials, by its original index (rel .w)
            const int e = __float_as_int(reinterpret_cast<const float*>(rel + at)[3]);
            float* dst = reinterpret_cast<float*>(partial + ((size_t)e * (size_t)pstride + (size_t)slot));
            dst[0] = k.ax[s];
            dst[1] = k.ay[s];
            dst[2] = k.az[s];
            if constexpr (DENS) dst[3] = k.aw[s];
        }
    }
}

// MINB = 2 allows 128 registers per thread (16 resident warps per SM);
// MINB = 3 caps them at 85 so 24 warps fit (the "lean" variant, for S <= 2).
template <int SMAX, int B, bool ADJ, int MINB, bool DENS>
__global__ void __launch_bounds__(256, MINB)
k_force(const BoxDev* __restrict__ boxes, const int* __restrict__ off, const float4* __restrict__ rel,
        const float4* __restrict__ gs, const int4* __restrict__ items, WsHeader* hdr,
        float4* __restrict__ partial, int pstride, int max_nseg)
{
    extern __shared__ __align__(16) unsigned char smem[];
    using W = WarpSmem<B, ADJ>;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char* w = smem + (size_t)wid * W::bytes(max_nseg);
    WarpBufs wb;
    wb.raw = reinterpret_cast<float4*>(w);
    wb.graw = reinterpret_cast<float4*>(w + W::raw_bytes);
    wb.soa = reinterpret_cast<float*>(w + W::raw_bytes + W::graw_bytes);
    wb.sh = reinterpret_cast<float2*>(w + W::raw_bytes + W::graw_bytes + W::soa_bytes);
    int* seg_pre = reinterpret_cast<int*>(w + W::raw_bytes + W::graw_bytes + W::soa_bytes + W::sh_bytes);
    int* seg_start = seg_pre + max_nseg + 1;
    float* seg_dy = reinterpret_cast<float*>(seg_start + max_nseg);
    float* seg_dz = seg_dy + max_nseg;

    const int n_items = *((volatile int*)&hdr->n_items);
    constexpr int CH = 32 * SMAX;

    for (;;) {
        int itn = 0;
        if (lane == 0) itn = atomicAdd(&hdr->queue, 1);
        itn = __shfl_sync(kFull, itn, 0);
        if (itn >= n_items) break;
        const int4 item = items[itn];
        const BoxDev& Bx = boxes[item.z];
        ItemCtx it;
        it.K = Bx.K;
        it.R = Bx.R;
        it.cb = Bx.cell_base;
        Coef cf;
        cf.c0 = Bx.c0;
        cf.c1 = Bx.c1;
        cf.c2 = Bx.c2;
        cf.e0 = Bx.e0;
        cf.e1 = Bx.e1;
        cf.eps2 = Bx.eps2;
        cf.dens_defer = Bx.dens_defer;
        const f2 b2 = pk(Bx.dens_b2, Bx.dens_b2);
        const int K = it.K, R = it.R;
        const int l = item.x - it.cb;
        it.i = l / (K * K);
        it.j = (l / K) % K;
        it.k = l % K;
        it.ns = 2 * R + 1;
        // sink cells (lanes 0..2R)
        it.sc_start = 0;
        it.sc_cnt = 0;
        if (lane < it.ns)
            it.sc_cnt = cell_count(off, it.cb + (wrap(it.i + lane - R, K) * K + it.j) * K + it.k,
                                   &it.sc_start);
        int incl = it.sc_cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        it.sc_incl = incl;
        it.n_sink = __shfl_sync(kFull, incl, it.ns - 1);
        it.chunk_begin = item.y * CH;
        // source segments: the plane's cells in rings around the centre (c_ring)
        const int nseg = it.ns * it.ns;
        int carry = 0;
        for (int base = 0; base < nseg; base += 32) {
            const int q = base + lane;
            int cnt = 0, st = 0, b = 0, d = 0;
            if (q < nseg) {
                b = c_ring[q][0];
                d = c_ring[q][1];
                cnt = cell_count(off, it.cb + (it.i * K + wrap(it.j + b, K)) * K + wrap(it.k + d, K), &st);
            }
            int inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc += y;
            }
            if (q < nseg) {
                seg_pre[q] = carry + inc - cnt;
                seg_start[q] = st;
                seg_dy[q] = (float)b;
                seg_dz[q] = (float)d;
            }
            carry += __shfl_sync(kFull, inc, 31);
        }
        if (lane == 0) seg_pre[nseg] = carry;
        it.n_src = carry;
        __syncwarp();
        it.n_c0 = seg_pre[1];
        it.n_near = seg_pre[nseg < 9 ? nseg : 9];
        const int n_chunk = min(CH, it.n_sink - it.chunk_begin);
        {
            const int c_cnt = __shfl_sync(kFull, it.sc_cnt, R);
            const int c_first = __shfl_sync(kFull, it.sc_incl, R) - c_cnt;  // pencil position of the centre cell
            it.has_self = c_cnt > 0 && it.chunk_begin < c_first + c_cnt && it.chunk_begin + n_chunk > c_first;
            // sinks of the cells R-1 .. R+1 of the pencil occupy positions [n_lo, n_hi)
            const int l0 = R > 0 ? R - 1 : 0, l1 = R > 0 ? R + 1 : 0;
            const int n_lo = __shfl_sync(kFull, it.sc_incl, l0) - __shfl_sync(kFull, it.sc_cnt, l0);
            const int n_hi = __shfl_sync(kFull, it.sc_incl, l1);
            it.near_x = it.chunk_begin < n_hi && it.chunk_begin + n_chunk > n_lo;
        }
        const int S = (n_chunk + 31) >> 5;  // <= SMAX
#define NF_RUN_ITEM(SS)                                                                                   \
    run_item<(SMAX >= SS ? SS : 1), B, ADJ, DENS>(it, cf, b2, rel, gs, wb, seg_pre, seg_start, seg_dy, seg_dz, \
                                                  partial, pstride, hdr)
        if (SMAX >= 8 && S == 8) NF_RUN_ITEM(8);
        else if (SMAX >= 7 && S == 7) NF_RUN_ITEM(7);
        else if (SMAX >= 6 && S == 6) NF_RUN_ITEM(6);
        else if (SMAX >= 5 && S == 5) NF_RUN_ITEM(5);
        else if (SMAX >= 4 && S == 4) NF_RUN_ITEM(4);
        else if (SMAX >= 3 && S == 3) NF_RUN_ITEM(3);
        else if (SMAX >= 2 && S == 2) NF_RUN_ITEM(2);
        else NF_RUN_ITEM(1);
#undef NF_RUN_ITEM
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Combine: per particle in input order, sum its row of 2R+1 partials without
// rounding error (FP32 TwoSum into a hi/lo pair), scale by a float-pair
// constant, round once; the optional net force is an FP64 sum
// ---------------------------------------------------------------------------

// Error-free sum of two floats: s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__global__ void __launch_bounds__(256)
k_combine(const BoxDev* __restrict__ boxes, int nboxes, const float4* __restrict__ partial, int pstride,
          float* __restrict__ out, float* __restrict__ rho, double* __restrict__ chunk_sums, bool adjoint)
{
    // block = one chunk of kCombineChunk particles (original order) of a single box;
    // a particle's 2R+1 partials are one contiguous row, so the loads and the
    // output rows of a warp are both contiguous
    __shared__ double red[3][8];
    int chunk = blockIdx.x;
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].chunk_base <= chunk) lo = mid;
        else hi = mid - 1;
    }
    const BoxDev& B = boxes[lo];
    const int nslot = 2 * B.R + 1;
    const double scale = adjoint ? B.scale_grad : B.scale_acc;
    // the scale as an unevaluated float pair: scale = s_hi + s_lo to ~2^-48
    const float s_hi = (float)scale;
    const float s_lo = (float)(scale - (double)s_hi);
    const double m = 1.0 / (double)B.N;
    const bool out_aligned8 = (reinterpret_cast<uintptr_t>(out) & 7) == 0;
    const int e0 = B.part_base + (chunk - B.chunk_base) * kCombineChunk;
    const int e1 = min(e0 + kCombineChunk, B.part_base + B.N);
    double net[3] = {0.0, 0.0, 0.0};
    constexpr int kMaxSlots = 2 * NF_MAX_R + 1;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const float4* row_in = partial + (size_t)e * (size_t)pstride;
        // issue every partial load first (they are independent), then sum
        float4 v[kMaxSlots];
#pragma unroll
        for (int q = 0; q < kMaxSlots; ++q) v[q] = q < nslot ? row_in[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        float a3[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // the 2R+1 pencil partials, summed without rounding error into (sh, sl)
            float sh = c == 0 ? v[0].x : (c == 1 ? v[0].y : v[0].z), sl = 0.0f;
#pragma unroll
            for (int q = 1; q < kMaxSlots; ++q) {
                if (q < nslot) {
                    const float x = c == 0 ? v[q].x : (c == 1 ? v[q].y : v[q].z);
                    float t, err;
                    two_sum(sh, x, t, err);
                    sh = t;
                    sl = __fadd_rn(sl, err);
                }
            }
            // (sh + sl) * (s_hi + s_lo), rounded once at the end
            const float p = __fmul_rn(sh, s_hi);
            const float perr = __fmaf_rn(sh, s_hi, -p);
            const float a = __fadd_rn(p, __fmaf_rn(sh, s_lo, __fmaf_rn(sl, s_hi, perr)));
            a3[c] = a;
            if (chunk_sums) net[c] += m * (double)a;
        }
        // the particle's row goes out in two stores (its 12 bytes start 8-byte
        // aligned for even e, 4 bytes past it for odd e)
        float* row = out + 3 * (size_t)e;
        if (out_aligned8 && (e & 1) == 0) {
            *reinterpret_cast<float2*>(row) = make_float2(a3[0], a3[1]);
            row[2] = a3[2];
        } else if (out_aligned8) {
            row[0] = a3[0];
            *reinterpret_cast<float2*>(row + 1) = make_float2(a3[1], a3[2]);
        } else {
            row[0] = a3[0];
            row[1] = a3[1];
            row[2] = a3[2];
        }
        if (rho) {
            // density partials (b^2 - r^2 sums), compensated, times 1/b^2
            float sh = v[0].w, sl = 0.0f;
#pragma unroll
            for (int q = 1; q < kMaxSlots; ++q) {
                if (q < nslot) {
                    float t, err;
                    two_sum(sh, v[q].w, t, err);
                    sh = t;
                    sl = __fadd_rn(sl, err);
                }
            }
            rho[e] = __fmul_rn(__fadd_rn(sh, sl), B.dens_inv_b2);
        }
    }
    if (chunk_sums) {
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double v = net[c];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
            if (lane == 0) red[c][w] = v;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            double v = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[threadIdx.x][q];
            chunk_sums[3 * (size_t)chunk + threadIdx.x] = v;
        }
    }
}

__global__ void k_net(const BoxDev* __restrict__ boxes, int nboxes, const double* __restrict__ chunk_sums,
                      double* __restrict__ net)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nboxes) return;
    const BoxDev& B = boxes[b];
    int n = (B.N + kCombineChunk - 1) / kCombineChunk;
    double v[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < n; ++q)
        for (int c = 0; c < 3; ++c) v[c] += chunk_sums[3 * (size_t)(B.chunk_base + q) + c];
    for (int c = 0; c < 3; ++c) net[3 * (size_t)b + c] = v[c];
}

int grid_for(size_t n, int threads)
{
    size_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535ull * 16) b = 65535ull * 16;
    return (int)b;
}

typedef void (*ForceKernel)(const BoxDev*, const int*, const float4*, const float4*, const int4*,
                            WsHeader*, float4*, int, int);

// The lean (85-register) variant is used when the tuning asks for 24 or more
// resident warps per SM.
bool wants_lean(const ForceTuning& t) { return t.sinks_per_lane <= 2 && t.warps_per_block * t.blocks_per_sm >= 24; }

template <bool ADJ, bool DENS>
ForceKernel pick_kernel(const ForceTuning& t)
{
    const int smax = t.sinks_per_lane, stage = t.stage;
    if (t.blocks_per_sm == 1 && stage == 128 && !DENS) {
        // one resident block of 8 warps per SM: the whole register file, so
        // three or four sinks per lane fit the adjoint without spills
        if (smax == 4) return k_force<4, 128, ADJ, 1, DENS>;
        if (smax == 3) return k_force<3, 128, ADJ, 1, DENS>;
    }
    if (wants_lean(t)) {
        if (stage == 128) {
            if (smax == 2) return k_force<2, 128, ADJ, 3, DENS>;
            if (smax == 1) return k_force<1, 128, ADJ, 3, DENS>;
        } else if (stage == 64) {
            if (smax == 2) return k_force<2, 64, ADJ, 3, DENS>;
            if (smax == 1) return k_force<1, 64, ADJ, 3, DENS>;
        }
        return nullptr;
    }
    if (stage == 128) {
        if (smax == 4) return k_force<4, 128, ADJ, 2, DENS>;
        if (smax == 3) return k_force<3, 128, ADJ, 2, DENS>;
        if (smax == 2) return k_force<2, 128, ADJ, 2, DENS>;
        if (smax == 1) return k_force<1, 128, ADJ, 2, DENS>;
    } else if (stage == 64) {
        if (smax == 4) return k_force<4, 64, ADJ, 2, DENS>;
        if (smax == 3) return k_force<3, 64, ADJ, 2, DENS>;
        if (smax == 2) return k_force<2, 64, ADJ, 2, DENS>;
        if (smax == 1) return k_force<1, 64, ADJ, 2, DENS>;
    }
    return nullptr;
}

ForceKernel pick(bool adjoint, bool density, const ForceTuning& t)
{
    if (adjoint) return pick_kernel<true, false>(t);
    return density ? pick_kernel<false, true>(t) : pick_kernel<false, false>(t);
}

size_t force_smem_bytes(bool adjoint, const ForceTuning& t, int max_nseg)
{
    size_t per = 0;
    if (t.stage == 128) per = adjoint ? WarpSmem<128, true>::bytes(max_nseg) : WarpSmem<128, false>::bytes(max_nseg);
    else per = adjoint ? WarpSmem<64, true>::bytes(max_nseg) : WarpSmem<64, false>::bytes(max_nseg);
    return per * (size_t)t.warps_per_block;
}

}  // namespace

bool force_tuning_supported(const ForceTuning& t)
{
    bool s_ok = t.sinks_per_lane >= 1 && t.sinks_per_lane <= 4;
    bool b_ok = t.stage == 64 || t.stage == 128;
    bool w_ok = t.warps_per_block == 4 || t.warps_per_block == 8;
    return s_ok && b_ok && w_ok && t.blocks_per_sm >= 0 && t.blocks_per_sm <= 8;
}

int force_blocks_per_sm(bool adjoint, bool density, const ForceTuning& t, int max_nseg)
{
    ForceKernel kfn = pick(adjoint, density, t);
    if (!kfn) return 0;
    size_t smem = force_smem_bytes(adjoint, t, max_nseg);
    if (ensure_smem((const void*)kfn, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)kfn, t.warps_per_block * 32, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_pencils(const BoxDev* boxes, int nboxes, int Ctot, const int* cell_off, int chunk, int stage,
                           int* chunks, unsigned* bucket_count, unsigned char* bucket_of, WsHeader* hdr,
                           cudaStream_t s)
{
    k_pencils<<<grid_for(Ctot, 256), 256, 0, s>>>(boxes, nboxes, Ctot, cell_off, chunk, stage, chunks,
                                                  bucket_count, bucket_of, hdr);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bucket_scan<<<1, kBuckets, 0, s>>>(bucket_count, hdr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_items(const BoxDev* boxes, int nboxes, int Ctot, const int* chunks,
                         const unsigned char* bucket_of, unsigned* bucket_count, int4* items,
                         WsHeader* hdr, cudaStream_t s)
{
    (void)hdr;
    k_items<<<grid_for(Ctot, 256), 256, 0, s>>>(boxes, nboxes, Ctot, chunks, bucket_of, bucket_count,
                                                items);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_g(const float* g, const int* perm, int Ntot, float4* gs, cudaStream_t s)
{
    k_gather_g<<<grid_for(Ntot, 256), 256, 0, s>>>(g, perm, Ntot, gs);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_force(bool adjoint, bool density, const ForceTuning& t, const BoxDev* boxes,
                         const int* cell_off, const float4* rel, const float4* gs, const int4* items,
                         WsHeader* hdr, float4* partial, int pstride, int max_nseg, cudaStream_t s)
{
    ForceKernel kfn = pick(adjoint, density, t);
    if (!kfn) return cudaErrorInvalidValue;
    size_t smem = force_smem_bytes(adjoint, t, max_nseg);
    cudaError_t e = ensure_smem((const void*)kfn, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)kfn, t.warps_per_block * 32, smem);
    if (e != cudaSuccess) return e;
    if (nb < 1) return cudaErrorInvalidConfiguration;
    if (t.blocks_per_sm > 0 && t.blocks_per_sm < nb) nb = t.blocks_per_sm;
    kfn<<<sms * nb, t.warps_per_block * 32, smem, s>>>(boxes, cell_off, rel, gs, items, hdr, partial, pstride,
                                                       max_nseg);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_combine(bool adjoint, const BoxDev* boxes, int nboxes, int nchunks, const float4* partial,
                           int pstride, float* out, float* rho, double* chunk_sums, cudaStream_t s)
{
    if (nchunks <= 0) return cudaSuccess;
    k_combine<<<nchunks, 256, 0, s>>>(boxes, nboxes, partial, pstride, out, rho, chunk_sums, adjoint);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_net(const BoxDev* boxes, int nboxes, const double* chunk_sums, double* net,
                       cudaStream_t s)
{
    k_net<<<(nboxes + 63) / 64, 64, 0, s>>>(boxes, nboxes, chunk_sums, net);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nf
