// C-ABI entry points of libnf: argument checks, workspace layout, launch order.
//
// Every entry point is a thin host function: it validates its arguments
// (nothing is enqueued when they are rejected), carves the caller's workspace
// into regions, and enqueues the kernels of nf_bin.cu and nf_force.cu on the
// caller's stream.  No entry point allocates memory or synchronises, except
// nf_status_read and nf_stats_read which read results back.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <map>
#include <mutex>
#include <utility>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "nf_internal.cuh"

namespace nf {

namespace {
std::atomic<long long> g_launches{0};
std::mutex g_smem_mutex;
std::map<std::pair<int, const void*>, int> g_smem_set;
}  // namespace

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaError_t ensure_smem(const void* fn, int bytes, bool max_carveout)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_smem_mutex);
    auto key = std::make_pair(dev, fn);
    auto it = g_smem_set.find(key);
    if (it != g_smem_set.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    // shared memory over L1 as far as it goes, so that occupancy is set by the
    // kernel's own limits
    if (e == cudaSuccess && max_carveout)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) g_smem_set[key] = bytes;
    return e;
}

namespace {

thread_local std::string g_last_error;

// Debug mode: guard blocks after every workspace region, filled when a call
// starts and checked when it ends (process-wide; off by default).
bool g_debug = false;

// Top-hat density: 0 = pick per box (deferred for b <= kDensDeferCells cell
// widths, fused above), 1 = always fused, 2 = always deferred.  Both modes
// give bit-identical results; the choice only moves work.
int g_dens_mode = 0;
constexpr double kDensDeferCells = 0.25;

struct GuardList {
    int count;
    long long off[24];
};

__global__ void k_guard_setup(void* ws, GuardList gl)
{
    WsHeader* h = static_cast<WsHeader*>(ws);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        h->guard_count = gl.count;
        for (int i = 0; i < gl.count; ++i) h->guard_off[i] = gl.off[i];
    }
    const int g = blockIdx.x;
    if (g < gl.count) {
        unsigned* w = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + gl.off[g]);
        for (int i = threadIdx.x; i < kGuardBytes / 4; i += blockDim.x) w[i] = kGuardWord;
    }
}

__global__ void k_guard_check(void* ws)
{
    WsHeader* h = static_cast<WsHeader*>(ws);
    const int n = h->guard_count;
    const int g = blockIdx.x;
    if (g >= n) return;
    const unsigned* w = reinterpret_cast<const unsigned*>(static_cast<const char*>(ws) + h->guard_off[g]);
    bool bad = false;
    for (int i = threadIdx.x; i < kGuardBytes / 4; i += blockDim.x) bad |= w[i] != kGuardWord;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&h->status, 1 << NF_ERR_CORRUPT);
}

// Per-stage profiling events of the last NF_PROFILE_RING calls (process-wide;
// off by default).  g_prof_count counts completed profiled calls.
bool g_profile_on = false;
long long g_prof_count = 0;
cudaEvent_t g_ev[NF_PROFILE_RING][5] = {};

cudaError_t prof_mark(int i, cudaStream_t s)
{
    if (!g_profile_on) return cudaSuccess;
    cudaEvent_t& ev = g_ev[g_prof_count % NF_PROFILE_RING][i];
    if (!ev) {
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
    }
    return cudaEventRecord(ev, s);
}
// Built-in tunings, measured best on GB300 (clustered 128^3 and 256^3 boxes):
// the forward four sinks per lane at 16 resident warps per SM; the adjoint
// (twice the registers per sink) four sinks per lane in the build for one
// block of 8 warps per SM, which has the whole register file (256^3: 147.1 ms
// against 152.3 ms for two sinks at 16 warps).
constexpr ForceTuning kBuiltinTuning = {4, 128, 8, 0};
constexpr ForceTuning kBuiltinTuningAdj = {4, 128, 8, 1};
ForceTuning g_default_tuning = kBuiltinTuning;
ForceTuning g_default_tuning_adj = kBuiltinTuningAdj;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* where)
{
    return fail(NF_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

constexpr double kEpsRatio = 2.16;  // eps_s / eps_p, Sec. "Force Softening"

struct Plan {
    int nboxes = 0;
    int64_t N = 0;       // total particles
    int64_t C = 0;       // total cells
    int64_t max_items = 0;
    int max_R = 1;
    int max_nseg = 9;
    int nchunks = 0;     // combine chunks
    SortPlan sp{};
    std::vector<BoxDev> boxes;
    // region offsets (bytes from ws)
    size_t o_boxes, o_keys_a, o_keys_b, o_rel_scratch, o_sort, o_off, o_rel, o_perm,
        o_chunks, o_bucket_of, o_bucket_count, o_items, o_gs, o_partial, o_chunk_sums, o_step, total;
    std::vector<size_t> guards;  // debug mode: guard block after each region
};

// Validates one box; fills the device constants.
int make_box(const nf_box& in, bool need_force, BoxDev* out)
{
    if (in.N < 1 || in.N >= (int64_t(1) << 31)) return fail(NF_ERR_ARG, "N = %lld out of [1, 2^31)", (long long)in.N);
    if (!(in.box > 0.0) || !std::isfinite(in.box)) return fail(NF_ERR_ARG, "box = %g must be finite and > 0", in.box);
    if (in.K < 1) return fail(NF_ERR_ARG, "K = %d must be >= 1", in.K);
    if ((int64_t)in.K * in.K * in.K >= (int64_t(1) << 31)) return fail(NF_ERR_ARG, "K^3 must be < 2^31 (K = %d)", in.K);
    BoxDev b;
    std::memset(&b, 0, sizeof b);
    b.K = in.K;
    b.R = in.R;
    b.N = (int)in.N;
    b.kl = (double)in.K / in.box;
    {
        // short dyadic form of kl: then x * kl is exact in FP64 for any FP32 x
        int e = 0;
        double f = std::frexp(b.kl, &e);                 // kl = f * 2^e, f in [0.5, 1)
        long long m = (long long)std::ldexp(f, 53);      // exact 53-bit integer
        int ex = e - 53;
        while (m > 0 && (m & 1) == 0) {
            m >>= 1;
            ++ex;
        }
        if (m > 0 && m < (1LL << 29)) {
            b.kl_mant = (int)m;
            b.kl_exp = ex;
            if (m == 1 && ex >= -100 && ex <= 100) b.kl_pow2 = (float)b.kl;
        }
    }
    const double w = in.box / in.K;
    b.scale_acc = 1.0 / ((double)in.N * w * w);
    b.scale_grad = 1.0 / ((double)in.N * w * w * w);
    if (need_force) {
        if (in.R < 1 || in.R > NF_MAX_R) return fail(NF_ERR_ARG, "R = %d out of [1, %d]", in.R, NF_MAX_R);
        if (in.K < 2 * in.R + 1)
            return fail(NF_ERR_ARG, "K = %d < 2R+1 = %d: the stencil would count a cell twice", in.K, 2 * in.R + 1);
        if (!(in.eps > 0.0) || !std::isfinite(in.eps)) return fail(NF_ERR_ARG, "eps = %g must be finite and > 0", in.eps);
        const double e = kEpsRatio * in.eps / w;  // eps_s in cell units
        if (e > in.R)
            return fail(NF_ERR_ARG, "eps_s = 2.16 eps = %g cells exceeds R = %d cells: the softening must end inside the near field", e, in.R);
        if (e < 1e-5) return fail(NF_ERR_ARG, "eps_s = %g cells is below 1e-5 cells", e);
        const double e2 = e * e, e3 = e2 * e, e4 = e3 * e, e5 = e4 * e;
        b.c0 = (float)(10.0 / e3);
        b.c1 = (float)(-15.0 / e4);
        b.c2 = (float)(6.0 / e5);
        b.e0 = (float)(-15.0 / e4);
        b.e1 = (float)(12.0 / e5);
        b.eps2 = (float)e2;
    }
    *out = b;
    return NF_OK;
}

int make_plan(const nf_box* boxes, int nboxes, bool need_force, int chunk_lanes, Plan* p)
{
    if (!boxes || nboxes < 1) return fail(NF_ERR_ARG, "need at least one box");
    p->nboxes = nboxes;
    p->boxes.resize(nboxes);
    int64_t N = 0, C = 0, items = 0, nchunks = 0;
    int max_R = 1;
    for (int b = 0; b < nboxes; ++b) {
        int rc = make_box(boxes[b], need_force, &p->boxes[b]);
        if (rc) {
            if (nboxes > 1) g_last_error = "box " + std::to_string(b) + ": " + g_last_error;
            return rc;
        }
        if (boxes[b].pos_offset != N)
            return fail(NF_ERR_ARG, "box %d: pos_offset = %lld, boxes must be packed back to back (expected %lld)", b,
                        (long long)boxes[b].pos_offset, (long long)N);
        BoxDev& d = p->boxes[b];
        d.part_base = (int)N;
        d.cell_base = (int)C;
        d.chunk_base = (int)nchunks;
        const int64_t cells = (int64_t)d.K * d.K * d.K;
        N += boxes[b].N;
        C += cells;
        nchunks += (boxes[b].N + kCombineChunk - 1) / kCombineChunk;
        if (need_force) {
            items += (2 * (int64_t)d.R + 1) * boxes[b].N / chunk_lanes + cells + 1;
            if (d.R > max_R) max_R = d.R;
        }
        if (N >= (int64_t(1) << 31)) return fail(NF_ERR_ARG, "total N must be < 2^31");
        if (C >= (int64_t(1) << 31) - 1) return fail(NF_ERR_ARG, "total cells must be < 2^31");
    }
    if (items >= (int64_t(1) << 31)) return fail(NF_ERR_ARG, "too many work items");
    p->N = N;
    p->C = C;
    p->max_items = items;
    p->max_R = max_R;
    p->max_nseg = (2 * max_R + 1) * (2 * max_R + 1);
    p->nchunks = (int)nchunks;
    p->sp = sort_plan(N, C);

    size_t o = 0;
    p->guards.clear();
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        if (g_debug) {
            p->guards.push_back(o);
            o = align_up(o + kGuardBytes);
        }
        return at;
    };
    take(sizeof(WsHeader));
    p->o_boxes = take(sizeof(BoxDev) * nboxes);
    p->o_keys_a = take(4 * (size_t)N);
    p->o_keys_b = take(4 * (size_t)N);
    p->o_rel_scratch = take(p->sp.passes > 1 ? 16 * (size_t)N : 16);
    p->o_sort = take(sort_ctl_bytes(p->sp));
    p->o_off = take(4 * (size_t)(C + 1));
    p->o_rel = take(16 * (size_t)N);
    p->o_perm = take(4 * (size_t)N);
    p->o_step = take(sizeof(StepScratch));
    if (need_force) {
        p->o_chunks = take(4 * (size_t)C);
        p->o_bucket_of = take((size_t)C);
        p->o_bucket_count = take(4 * kBuckets);
        p->o_items = take(16 * (size_t)items);
        p->o_gs = take(16 * (size_t)N);
        p->o_partial = take(4 * 4 * (size_t)(2 * max_R + 1) * (size_t)N);
        p->o_chunk_sums = take(8 * 3 * (size_t)nchunks);
    } else {
        p->o_chunks = p->o_bucket_of = p->o_bucket_count = p->o_items = p->o_gs = p->o_partial =
            p->o_chunk_sums = 0;
    }
    p->total = o;
    return NF_OK;
}

template <typename T>
T* at(void* ws, size_t off)
{
    return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

int check_tuning(const nf_tuning* t, ForceTuning* out, bool adjoint = false)
{
    if (!t) {
        *out = adjoint ? g_default_tuning_adj : g_default_tuning;
        return NF_OK;
    }
    ForceTuning f = {t->sinks_per_lane, t->stage, t->warps_per_block, t->blocks_per_sm};
    if (!force_tuning_supported(f))
        return fail(NF_ERR_ARG, "unsupported tuning (sinks_per_lane %d, stage %d, warps %d, blocks %d)",
                    t->sinks_per_lane, t->stage, t->warps_per_block, t->blocks_per_sm);
    *out = f;
    return NF_OK;
}

#define NF_CUDA(call, where)                                  \
    do {                                                      \
        cudaError_t e__ = (call);                             \
        if (e__ != cudaSuccess) return cuda_fail(e__, where); \
    } while (0)

// Clears the header, uploads the box table, bins every particle.
// Debug mode: check every guard block of the workspace at the end of a call.
int finish_call(void* ws, cudaStream_t s)
{
    if (!g_debug) return NF_OK;
    k_guard_check<<<24, 64, 0, s>>>(ws);
    count_launches(1);
    NF_CUDA(cudaGetLastError(), "guard check");
    return NF_OK;
}

// Clears the status header of a workspace and, in debug mode, fills its guard
// blocks and records them in the header (every call that later runs
// finish_call on the workspace starts with this).
int init_ws(const Plan& p, void* ws, cudaStream_t s)
{
    NF_CUDA(cudaMemsetAsync(at<WsHeader>(ws, 0), 0, sizeof(WsHeader), s), "clear header");
    if (g_debug && !p.guards.empty()) {
        GuardList gl;
        std::memset(&gl, 0, sizeof gl);
        gl.count = (int)std::min<size_t>(p.guards.size(), 24);
        for (int i = 0; i < gl.count; ++i) gl.off[i] = (long long)p.guards[i];
        k_guard_setup<<<gl.count, 64, 0, s>>>(ws, gl);
        count_launches(1);
        NF_CUDA(cudaGetLastError(), "guard setup");
    }
    return NF_OK;
}

int run_binning(const Plan& p, const float* pos, void* ws, int32_t* cell_off, float4* rel, int32_t* perm,
                cudaStream_t s)
{
    WsHeader* hdr = at<WsHeader>(ws, 0);
    BoxDev* boxes = at<BoxDev>(ws, p.o_boxes);
    int rc = init_ws(p, ws, s);
    if (rc) return rc;
    for (int first = 0; first < p.nboxes; first += kMaxBoxesPerFill) {
        BoxFill f;
        std::memset(&f, 0, sizeof f);
        f.first = first;
        f.count = std::min(kMaxBoxesPerFill, p.nboxes - first);
        for (int q = 0; q < f.count; ++q) f.b[q] = p.boxes[first + q];
        NF_CUDA(launch_fill_boxes(f, boxes, s), "box table");
    }
    NF_CUDA(run_sort(p.sp, pos, (int)p.N, (int)p.C, boxes, p.nboxes, at<void>(ws, p.o_sort),
                     at<float4>(ws, p.o_rel_scratch), at<int>(ws, p.o_keys_a), at<int>(ws, p.o_keys_b), rel, perm,
                     cell_off, hdr, s),
            "binning sort");
    return NF_OK;
}

int run_forces(const Plan& p, bool adjoint, const ForceTuning& t, const float* pos, const float* g, float* out,
               double* net, float* rho, void* ws, cudaStream_t s)
{
    WsHeader* hdr = at<WsHeader>(ws, 0);
    BoxDev* boxes = at<BoxDev>(ws, p.o_boxes);
    int32_t* off = at<int32_t>(ws, p.o_off);
    float4* rel = at<float4>(ws, p.o_rel);
    int32_t* perm = at<int32_t>(ws, p.o_perm);
    NF_CUDA(prof_mark(0, s), "profile");
    int rc = run_binning(p, pos, ws, off, rel, perm, s);
    if (rc) return rc;
    NF_CUDA(prof_mark(1, s), "profile");
    unsigned* bucket_count = at<unsigned>(ws, p.o_bucket_count);
    NF_CUDA(cudaMemsetAsync(bucket_count, 0, 4 * kBuckets, s), "clear buckets");
    const int CH = 32 * t.sinks_per_lane;
    NF_CUDA(launch_pencils(boxes, p.nboxes, (int)p.C, off, CH, t.stage, at<int>(ws, p.o_chunks), bucket_count,
                           at<unsigned char>(ws, p.o_bucket_of), hdr, s),
            "pencils");
    NF_CUDA(launch_items(boxes, p.nboxes, (int)p.C, at<int>(ws, p.o_chunks), at<unsigned char>(ws, p.o_bucket_of),
                         bucket_count, at<int4>(ws, p.o_items), hdr, s),
            "work items");
    float4* gs = at<float4>(ws, p.o_gs);
    if (adjoint) NF_CUDA(launch_gather_g(g, perm, (int)p.N, gs, s), "gather g");
    float4* partial = at<float4>(ws, p.o_partial);
    const int pstride = 2 * p.max_R + 1;  // partial row of a particle: one float4 per pencil slot
    NF_CUDA(prof_mark(2, s), "profile");
    NF_CUDA(launch_force(adjoint, rho != nullptr, t, boxes, off, rel, gs, at<int4>(ws, p.o_items), hdr, partial,
                         pstride, p.max_nseg, s),
            adjoint ? "adjoint kernel" : "force kernel");
    NF_CUDA(prof_mark(3, s), "profile");
    double* chunk_sums = net ? at<double>(ws, p.o_chunk_sums) : nullptr;
    NF_CUDA(launch_combine(adjoint, boxes, p.nboxes, p.nchunks, partial, pstride, out, rho, chunk_sums, s),
            "combine");
    if (net) NF_CUDA(launch_net(boxes, p.nboxes, chunk_sums, net, s), "net force");
    NF_CUDA(prof_mark(4, s), "profile");
    if (g_profile_on) ++g_prof_count;
    return finish_call(ws, s);
}

int check_ws(const Plan& p, void* ws, size_t ws_bytes)
{
    if (!ws) return fail(NF_ERR_WORKSPACE, "workspace is NULL");
    if ((reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0)
        return fail(NF_ERR_WORKSPACE, "workspace must be %zu-byte aligned", kAlign);
    if (ws_bytes < p.total)
        return fail(NF_ERR_WORKSPACE, "workspace too small: %zu bytes given, %zu needed", ws_bytes, p.total);
    return NF_OK;
}

nf_box one_box(int64_t N, double box, int K, int R, double eps)
{
    nf_box b;
    b.N = N;
    b.pos_offset = 0;
    b.box = box;
    b.eps = eps;
    b.K = K;
    b.R = R;
    return b;
}

int forces_entry(const nf_box* boxes, int nboxes, bool adjoint, const float* pos, const float* g, float* out,
                 double* net, const nf_tuning* tune, void* ws, size_t ws_bytes, void* stream,
                 double dens_b = 0.0, float* rho = nullptr)
{
    g_last_error.clear();
    ForceTuning t;
    int rc = check_tuning(tune, &t, adjoint);
    if (rc) return rc;
    Plan p;
    rc = make_plan(boxes, nboxes, true, 32 * t.sinks_per_lane, &p);
    if (rc) return rc;
    if (!pos || !out || (adjoint && !g)) return fail(NF_ERR_ARG, "null pointer argument");
    if (rho) {
        for (int b = 0; b < nboxes; ++b) {
            const double w = boxes[b].box / boxes[b].K;
            if (!(dens_b > 0.0) || !std::isfinite(dens_b) || dens_b > boxes[b].R * w)
                return fail(NF_ERR_ARG, "density radius b = %g must be in (0, R w = %g]: the top hat must lie in the near field",
                            dens_b, boxes[b].R * w);
            const double bc = dens_b / w;
            p.boxes[b].dens_b2 = (float)(bc * bc);
            p.boxes[b].dens_inv_b2 = (float)(1.0 / (bc * bc));
            p.boxes[b].dens_defer = g_dens_mode == 2 || (g_dens_mode == 0 && bc <= kDensDeferCells);
        }
    }
    rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    return run_forces(p, adjoint, t, pos, g, out, net, rho, ws, static_cast<cudaStream_t>(stream));
}

}  // namespace
}  // namespace nf

namespace nf {
namespace {

// Scratch of nf_forces_noalloc: a fixed array in every loaded device image.
// Host code must not pass this name to a kernel (on the host it is only a
// stand-in); its device address comes from cudaGetSymbolAddress, looked up
// once per device with that device current and then reused.
constexpr int kMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NF_NOALLOC_SCRATCH_BYTES];
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "nf_forces_noalloc: current device");
    if (dev < 0 || dev >= kMaxDevices) return fail(NF_ERR_ARG, "nf_forces_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "nf_forces_noalloc: scratch address");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return NF_OK;
}

}  // namespace
}  // namespace nf

using namespace nf;

extern "C" {

const char* nf_last_error(void) { return g_last_error.c_str(); }

const char* nf_version(void) { return "nf 0.1 (sm_103a)"; }

size_t nf_workspace_bytes(int64_t N, int K, int R)
{
    // the size does not depend on box or eps: use box 1 and a valid softening
    nf_box b = one_box(N, 1.0, K, R, K > 0 ? 0.5 / (kEpsRatio * K) : 1.0);
    Plan p;
    if (make_plan(&b, 1, true, 32, &p)) return 0;
    return p.total;
}

size_t nf_workspace_bytes_batched(const nf_box* boxes, int nboxes)
{
    Plan p;
    if (make_plan(boxes, nboxes, true, 32, &p)) return 0;
    return p.total;
}

int nf_bin(const float* pos, int64_t N, double box, int K, int32_t* cell_offsets, float* rel, int32_t* perm,
           void* ws, size_t ws_bytes, void* stream)
{
    g_last_error.clear();
    nf_box b = one_box(N, box, K, 0, 0.0);
    Plan p;
    int rc = make_plan(&b, 1, false, 32, &p);
    if (rc) return rc;
    if (!pos || !cell_offsets || !rel || !perm) return fail(NF_ERR_ARG, "null pointer argument");
    if ((reinterpret_cast<uintptr_t>(rel) & 15) != 0) return fail(NF_ERR_ARG, "rel must be 16-byte aligned");
    // nf_bin needs only the binning regions, which precede the force regions
    rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    rc = run_binning(p, pos, ws, cell_offsets, reinterpret_cast<float4*>(rel), perm, static_cast<cudaStream_t>(stream));
    if (rc) return rc;
    return finish_call(ws, static_cast<cudaStream_t>(stream));
}

int nf_forces(const float* pos, int64_t N, double box, int K, int R, double eps, float* acc, double* net, void* ws,
              size_t ws_bytes, void* stream)
{
    nf_box b = one_box(N, box, K, R, eps);
    return forces_entry(&b, 1, false, pos, nullptr, acc, net, nullptr, ws, ws_bytes, stream);
}

int nf_forces_density(const float* pos, int64_t N, double box, int K, int R, double eps, double b, float* acc,
                      float* rho, void* ws, size_t ws_bytes, void* stream)
{
    if (!rho) {
        g_last_error.clear();
        return fail(NF_ERR_ARG, "null pointer argument");
    }
    nf_box bx = one_box(N, box, K, R, eps);
    return forces_entry(&bx, 1, false, pos, nullptr, acc, nullptr, nullptr, ws, ws_bytes, stream, b, rho);
}

int nf_forces_adjoint(const float* pos, const float* g, int64_t N, double box, int K, int R, double eps, float* grad,
                      void* ws, size_t ws_bytes, void* stream)
{
    nf_box b = one_box(N, box, K, R, eps);
    return forces_entry(&b, 1, true, pos, g, grad, nullptr, nullptr, ws, ws_bytes, stream);
}

int nf_forces_batched(const nf_box* boxes, int nboxes, const float* pos_cat, float* acc_cat, double* net,
                      const nf_tuning* tune, void* ws, size_t ws_bytes, void* stream)
{
    return forces_entry(boxes, nboxes, false, pos_cat, nullptr, acc_cat, net, tune, ws, ws_bytes, stream);
}

int nf_forces_adjoint_batched(const nf_box* boxes, int nboxes, const float* pos_cat, const float* g_cat,
                              float* grad_cat, const nf_tuning* tune, void* ws, size_t ws_bytes, void* stream)
{
    return forces_entry(boxes, nboxes, true, pos_cat, g_cat, grad_cat, nullptr, tune, ws, ws_bytes, stream);
}

int nf_set_default_tuning(const nf_tuning* t)
{
    g_last_error.clear();
    if (!t) {
        g_default_tuning = kBuiltinTuning;
        g_default_tuning_adj = kBuiltinTuningAdj;
        return NF_OK;
    }
    ForceTuning f;
    int rc = check_tuning(t, &f);
    if (rc) return rc;
    g_default_tuning = f;
    g_default_tuning_adj = f;
    return NF_OK;
}

int nf_set_default_tuning_adjoint(const nf_tuning* t)
{
    g_last_error.clear();
    if (!t) {
        g_default_tuning_adj = kBuiltinTuningAdj;
        return NF_OK;
    }
    ForceTuning f;
    int rc = check_tuning(t, &f);
    if (rc) return rc;
    g_default_tuning_adj = f;
    return NF_OK;
}

static void copy_tuning(const ForceTuning& f, nf_tuning* t)
{
    t->sinks_per_lane = f.sinks_per_lane;
    t->stage = f.stage;
    t->warps_per_block = f.warps_per_block;
    t->blocks_per_sm = f.blocks_per_sm;
}

void nf_get_default_tuning(nf_tuning* t)
{
    if (t) copy_tuning(g_default_tuning, t);
}

void nf_get_default_tuning_adjoint(nf_tuning* t)
{
    if (t) copy_tuning(g_default_tuning_adj, t);
}

int nf_forces_noalloc(const float* pos, int64_t N, double box, int K, int R, double eps, float* acc, double* net,
                      void* stream)
{
    g_last_error.clear();
    // Host-side checks first: nothing touches the device for a rejected call.
    nf_box b = one_box(N, box, K, R, eps);
    ForceTuning t;
    int rc = check_tuning(nullptr, &t);
    if (rc) return rc;
    Plan p;
    rc = make_plan(&b, 1, true, 32 * t.sinks_per_lane, &p);
    if (rc) return rc;
    if (!pos || !acc) return fail(NF_ERR_ARG, "null pointer argument");
    if (p.total > (size_t)NF_NOALLOC_SCRATCH_BYTES)
        return fail(NF_ERR_WORKSPACE,
                    "nf_forces_noalloc: N = %lld, K = %d, R = %d needs %zu bytes of scratch, more than the "
                    "library's fixed %u-byte array; call nf_forces with a workspace instead",
                    (long long)N, K, R, p.total, (unsigned)NF_NOALLOC_SCRATCH_BYTES);
    void* scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    return forces_entry(&b, 1, false, pos, nullptr, acc, net, nullptr, scratch, NF_NOALLOC_SCRATCH_BYTES,
                        stream);
}

int nf_timestep(const float* pos, const float* vel, const float* acc, int64_t N, double box, int K,
                const nf_step_params* prm, double* dt, void* ws, size_t ws_bytes, void* stream)
{
    g_last_error.clear();
    nf_box b = one_box(N, box, K, 0, 0.0);
    Plan p;
    int rc = make_plan(&b, 1, false, 32, &p);
    if (rc) return rc;
    if (!pos || !vel || !acc || !dt || !prm) return fail(NF_ERR_ARG, "null pointer argument");
    if (!(prm->eta_acc > 0.0) || !(prm->hubble >= 0.0) || (prm->hubble > 0.0 && !(prm->eta_h > 0.0)))
        return fail(NF_ERR_ARG, "step parameters need eta_acc > 0, hubble >= 0 and eta_h > 0 when hubble > 0");
    rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t* off = at<int32_t>(ws, p.o_off);
    int32_t* perm = at<int32_t>(ws, p.o_perm);
    rc = run_binning(p, pos, ws, off, at<float4>(ws, p.o_rel), perm, s);
    if (rc) return rc;
    NF_CUDA(launch_timestep(off, perm, vel, acc, (int)p.C, (long long)N, prm->eta_acc, prm->eta_h, prm->hubble,
                            at<StepScratch>(ws, p.o_step), dt, s),
            "time step");
    return finish_call(ws, s);
}

int nf_kdk_step(float* pos, float* vel, float* acc, int64_t N, double box, int K, int R, double eps, double* dt,
                const nf_step_params* prm, void* ws, size_t ws_bytes, void* stream)
{
    g_last_error.clear();
    nf_box b = one_box(N, box, K, R, eps);
    ForceTuning t;
    int rc = check_tuning(nullptr, &t);
    if (rc) return rc;
    Plan p;
    rc = make_plan(&b, 1, true, 32 * t.sinks_per_lane, &p);
    if (rc) return rc;
    if (!pos || !vel || !acc || !dt) return fail(NF_ERR_ARG, "null pointer argument");
    if (prm && (!(prm->eta_acc > 0.0) || !(prm->hubble >= 0.0) || (prm->hubble > 0.0 && !(prm->eta_h > 0.0))))
        return fail(NF_ERR_ARG, "step parameters need eta_acc > 0, hubble >= 0 and eta_h > 0 when hubble > 0");
    rc = check_ws(p, ws, ws_bytes);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    NF_CUDA(launch_kick(vel, acc, (int)N, dt, 0.5, s), "kick");
    NF_CUDA(launch_drift(pos, vel, (int)N, dt, (float)box, s), "drift");
    rc = run_forces(p, false, t, pos, nullptr, acc, nullptr, nullptr, ws, s);
    if (rc) return rc;
    NF_CUDA(launch_kick(vel, acc, (int)N, dt, 0.5, s), "kick");
    if (prm)
        NF_CUDA(launch_timestep(at<int32_t>(ws, p.o_off), at<int32_t>(ws, p.o_perm), vel, acc, (int)p.C, (long long)N,
                                prm->eta_acc, prm->eta_h, prm->hubble, at<StepScratch>(ws, p.o_step), dt, s),
                "time step");
    return finish_call(ws, s);
}

int nf_multipoles(const float* pos, int64_t N, double box, int K, int p, double* M, void* ws, size_t ws_bytes,
                  void* stream)
{
    g_last_error.clear();
    nf_box b = one_box(N, box, K, 0, 0.0);
    Plan pl;
    int rc = make_plan(&b, 1, false, 32, &pl);
    if (rc) return rc;
    if (p < 0 || p > NF_MAX_MULTIPOLE_ORDER) return fail(NF_ERR_ARG, "multipole order p = %d out of [0, %d]", p, NF_MAX_MULTIPOLE_ORDER);
    if (!pos || !M) return fail(NF_ERR_ARG, "null pointer argument");
    rc = check_ws(pl, ws, ws_bytes);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t* off = at<int32_t>(ws, pl.o_off);
    float4* rel = at<float4>(ws, pl.o_rel);
    rc = run_binning(pl, pos, ws, off, rel, at<int32_t>(ws, pl.o_perm), s);
    if (rc) return rc;
    NF_CUDA(launch_multipoles(off, rel, (int)pl.C, box / K, p, M, s), "multipoles");
    return finish_call(ws, s);
}

// ---- far field -------------------------------------------------------------

namespace {

// Ewald split of the derivatives tensor: alpha * box, real-space images
// n in [-1, 1]^3 around the centred offset, reciprocal vectors |h_i| <= 14.
// With these the left-out terms are below 1e-20 of the kept ones up to order 12.
constexpr double kFarAlphaL = 5.0;
constexpr int kFarNimg = 1;
constexpr int kFarHmax = 14;

struct DerivLayout {
    int nt = 0, nr = 0;
    long long npairs = 0, nnz = 0;
    size_t o_seg = 0, o_pairs = 0, o_dh = 0, o_rseg = 0, o_rk = 0, o_rcoef = 0, o_ops = 0, o_opf = 0, total = 0;
    size_t o_drdf = 0, o_pcdf = 0, o_tw = 0;  // double-float path: derivatives, pair coefficients, twiddles
    size_t o_tw64 = 0;                        // FP64 twiddles
};

// K^3 and n_t K^3 below 2^31 (32-bit field offsets)
bool far_args_ok(int K, int p)
{
    if (K < 1 || p < 0 || p > NF_MAX_FAR_ORDER) return false;
    const int64_t cells = (int64_t)K * K * K;
    return cells < (int64_t(1) << 31) && (int64_t)far_terms_host(p) * cells < (int64_t(1) << 31);
}

// Table sizes of order p (they do not depend on the cell width), cached.
struct TableCounts {
    int nr;
    long long npairs, nnz;
};
TableCounts table_counts(int p)
{
    static std::mutex mu;
    static std::map<int, TableCounts> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(p);
    if (it != cache.end()) return it->second;
    const FarTables tb = far_tables(p, 1.0);
    const TableCounts c{tb.nr, (long long)tb.pairs.size(), (long long)tb.red_k.size()};
    cache[p] = c;
    return c;
}

DerivLayout deriv_layout(int K, int p)
{
    DerivLayout L;
    L.nt = far_terms_host(p);
    const TableCounts c = table_counts(p);
    L.nr = c.nr;
    L.npairs = c.npairs;
    L.nnz = c.nnz;
    size_t o = align_up(sizeof(DerivHeader));
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    L.o_seg = take(4 * (size_t)(L.nr + 1));
    L.o_pairs = take(sizeof(FarPair) * (size_t)L.npairs);
    L.o_rseg = take(4 * (size_t)(L.nr + 1));
    L.o_rk = take(4 * (size_t)L.nnz);
    L.o_rcoef = take(8 * (size_t)L.nnz);
    L.o_ops = take(sizeof(int4) * (size_t)L.nt);
    L.o_opf = take(sizeof(double2) * (size_t)L.nt);
    L.o_dh = take(8 * (size_t)L.nt * K * K * (K / 2 + 1));  // one real per (term, frequency)
    L.o_drdf = take(8 * (size_t)L.nt * K * K * (K / 2 + 1));  // the same as double-float pairs
    L.o_pcdf = take(8 * (size_t)L.npairs);
    L.o_tw = take(16 * (size_t)K);
    L.o_tw64 = take(16 * (size_t)K);
    L.total = o;
    return L;
}

struct FarLayout {
    size_t o_M = 0, o_Mr = 0, o_Mh = 0, o_Th = 0, o_Tdf = 0, o_m002 = 0, o_s002 = 0, total = 0;
};

// The far-field regions follow the binning plan's; in debug mode each is
// followed by a guard block like the plan's regions (appended to guards).
// M: complete multipoles (FP64 mode), later the rebuilt FP64 Taylors [C][nt];
// Mr: reduced multipoles, later the reduced Taylors [C][nr], 8 bytes each
// (FP64, or a double-float pair on the double-float transform path); Mh, Th:
// spectra [nr][nq], 16 bytes each (FP64 complex or double-float complex);
// Tdf: double-float Taylor pairs [C][nt]; m002: each cell's (0,0,2)
// multipole [C]; s002: partial sums of the (0,0,2) multipoles.
FarLayout far_layout(const Plan& pl, int K, int p, std::vector<size_t>* guards = nullptr)
{
    FarLayout F;
    const int nt = far_terms_host(p), nr = table_counts(p).nr;
    const size_t cells = (size_t)K * K * K;
    const size_t spec = 16 * (size_t)nr * K * K * (K / 2 + 1);
    size_t o = align_up(pl.total);
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        if (g_debug) {
            if (guards) guards->push_back(o);
            o = align_up(o + kGuardBytes);
        }
        return at;
    };
    F.o_M = take(8 * (size_t)nt * cells);
    F.o_Mr = take(8 * (size_t)nr * cells);
    F.o_Mh = take(spec);
    F.o_Th = take(spec);
    F.o_Tdf = take(8 * (size_t)nt * cells);
    F.o_m002 = take(8 * cells);
    F.o_s002 = take(8 * (size_t)far_sum_partials());
    F.total = o;
    return F;
}

struct DerivKey {
    int K, R, p;
    double box;
};
// Arithmetic of the per-particle far-field kernels (multipoles, Taylor
// evaluation): NF_FAR_DOUBLE_FLOAT or NF_FAR_FP64; process-wide.
std::atomic<int> g_far_arith{NF_FAR_DOUBLE_FLOAT};
std::mutex g_deriv_mu;
std::map<const void*, DerivKey> g_derivs;

int far_validate(int K, int R, int p, double box)
{
    if (!far_args_ok(K, p))
        return fail(NF_ERR_ARG, "far field: K = %d or order p = %d out of range (p <= %d, (p+3)(p+2)(p+1)/6 K^3 < 2^31)",
                    K, p, NF_MAX_FAR_ORDER);
    if (R < 1 || R > NF_MAX_R) return fail(NF_ERR_ARG, "R = %d out of [1, %d]", R, NF_MAX_R);
    if (K < 2 * R + 1) return fail(NF_ERR_ARG, "K = %d < 2R+1 = %d: the stencil would wrap onto itself", K, 2 * R + 1);
    if (!(box > 0.0) || !std::isfinite(box)) return fail(NF_ERR_ARG, "box = %g must be finite and > 0", box);
    return NF_OK;
}

}  // namespace

namespace {


}  // namespace

int nf_far_set_arith(int mode)
{
    g_last_error.clear();
    if (mode != NF_FAR_FP64 && mode != NF_FAR_DOUBLE_FLOAT)
        return fail(NF_ERR_ARG, "far-field arithmetic %d is neither NF_FAR_FP64 nor NF_FAR_DOUBLE_FLOAT", mode);
    g_far_arith.store(mode);
    return NF_OK;
}

int nf_far_get_arith(void) { return g_far_arith.load(); }

int nf_far_release(void)
{
    g_last_error.clear();
    return NF_OK;  // the library keeps no transform plans (its transforms are its own kernels)
}

size_t nf_derivatives_bytes(int K, int p)
{
    if (!far_args_ok(K, p)) return 0;
    return deriv_layout(K, p).total;
}

size_t nf_far_workspace_bytes(int64_t N, int K, int p)
{
    if (!far_args_ok(K, p)) return 0;
    nf_box b = one_box(N, 1.0, K, 0, 0.0);
    Plan pl;
    if (make_plan(&b, 1, false, 32, &pl)) return 0;
    return far_layout(pl, K, p).total;
}

int nf_derivatives(int K, int R, int p, double box, void* derivs, size_t derivs_bytes, void* ws, size_t ws_bytes,
                   void* stream)
{
    g_last_error.clear();
    int rc = far_validate(K, R, p, box);
    if (rc) return rc;
    if (!derivs) return fail(NF_ERR_ARG, "derivs is NULL");
    const DerivLayout L = deriv_layout(K, p);
    if ((reinterpret_cast<uintptr_t>(derivs) & (kAlign - 1)) != 0)
        return fail(NF_ERR_WORKSPACE, "derivs must be %zu-byte aligned", kAlign);
    if (derivs_bytes < L.total)
        return fail(NF_ERR_WORKSPACE, "derivs too small: %zu bytes given, %zu needed", derivs_bytes, L.total);
    nf_box b = one_box(1, box, K, 0, 0.0);
    Plan pl;
    rc = make_plan(&b, 1, false, 32, &pl);
    if (rc) return rc;
    const FarLayout F = far_layout(pl, K, p);
    if (!ws) return fail(NF_ERR_WORKSPACE, "workspace is NULL");
    if ((reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0)
        return fail(NF_ERR_WORKSPACE, "workspace must be %zu-byte aligned", kAlign);
    if (ws_bytes < F.total)
        return fail(NF_ERR_WORKSPACE, "workspace too small: %zu bytes given, %zu needed", ws_bytes, F.total);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double alpha = kFarAlphaL / box;
    // D (real, [C][nt]) in the multipole region; its spectrum ([nt][nq] complex) needs
    // 16 nt nq bytes: the multipole, reduced and double-float regions that follow
    // the first one are contiguous and large enough (checked below)
    double* D = at<double>(ws, F.o_M);
    double2* Dh = at<double2>(ws, F.o_Mr);
    if (F.o_Mr + 16 * (size_t)L.nt * K * K * (K / 2 + 1) > F.total)
        return fail(NF_ERR_WORKSPACE, "internal: derivative spectrum does not fit the far workspace");
    {
        // the FP64 twiddles first: the derivatives' transform below reads them
        const std::vector<double2> tw64 = far_twiddles64(K);
        NF_CUDA(cudaMemcpyAsync(at<char>(derivs, L.o_tw64), tw64.data(), sizeof(double2) * tw64.size(),
                                cudaMemcpyHostToDevice, s),
                "far tables");
    }
    NF_CUDA(launch_deriv_real(K, R, p, box, alpha, kFarNimg, D, s), "derivatives (real space)");
    NF_CUDA(launch_far_fft64(K, L.nt, true, D, Dh, nullptr, at<double2>(derivs, L.o_tw64), s),
            "derivatives (forward transform)");
    NF_CUDA(launch_deriv_recip(K, p, box, alpha, kFarHmax, Dh, at<double>(derivs, L.o_dh), s),
            "derivatives (reciprocal space)");
    {
        // the fold, reduced-pair and rebuild tables, built on the host (pageable copies:
        // the call returns once the data is staged)
        const FarTables tb = far_tables(p, box / K);
        if ((long long)tb.pairs.size() != L.npairs || (long long)tb.red_k.size() != L.nnz || tb.nr != L.nr)
            return fail(NF_ERR_ARG, "internal: far-field table sizes disagree");
        auto up = [&](size_t off, const void* src, size_t bytes) {
            return bytes ? cudaMemcpyAsync(at<char>(derivs, off), src, bytes, cudaMemcpyHostToDevice, s)
                         : cudaSuccess;
        };
        NF_CUDA(up(L.o_seg, tb.pair_seg.data(), 4 * tb.pair_seg.size()), "far tables");
        NF_CUDA(up(L.o_pairs, tb.pairs.data(), sizeof(FarPair) * tb.pairs.size()), "far tables");
        NF_CUDA(up(L.o_rseg, tb.red_seg.data(), 4 * tb.red_seg.size()), "far tables");
        NF_CUDA(up(L.o_rk, tb.red_k.data(), 4 * tb.red_k.size()), "far tables");
        NF_CUDA(up(L.o_rcoef, tb.red_coef.data(), 8 * tb.red_coef.size()), "far tables");
        NF_CUDA(up(L.o_ops, tb.ops.data(), sizeof(int4) * tb.ops.size()), "far tables");
        NF_CUDA(up(L.o_opf, tb.opf.data(), sizeof(double2) * tb.opf.size()), "far tables");
        {
            const std::vector<float4> tw = far_twiddles(K);
            NF_CUDA(up(L.o_pcdf, tb.pair_cdf.data(), sizeof(float2) * tb.pair_cdf.size()), "far tables");
            NF_CUDA(up(L.o_tw, tw.data(), sizeof(float4) * tw.size()), "far tables");
            NF_CUDA(launch_to_df(at<double>(derivs, L.o_dh), (long long)L.nt * K * K * (K / 2 + 1),
                                 at<void>(derivs, L.o_drdf), s),
                    "derivatives (double-float copy)");
        }
    }
    DerivHeader h;
    std::memset(&h, 0, sizeof h);
    h.magic = kDerivMagic;
    h.K = K;
    h.R = R;
    h.p = p;
    h.box = box;
    h.alpha = alpha;
    h.nimg = kFarNimg;
    h.hmax = kFarHmax;
    h.nt = L.nt;
    h.nr = L.nr;
    h.npairs = L.npairs;
    h.nnz = L.nnz;
    h.o_seg = L.o_seg;
    h.o_pairs = L.o_pairs;
    h.o_dh = L.o_dh;
    h.o_rseg = L.o_rseg;
    h.o_rk = L.o_rk;
    h.o_rcoef = L.o_rcoef;
    h.o_ops = L.o_ops;
    h.o_opf = L.o_opf;
    h.o_drdf = L.o_drdf;
    h.o_pcdf = L.o_pcdf;
    h.o_tw = L.o_tw;
    h.o_tw64 = L.o_tw64;
    h.total = L.total;
    NF_CUDA(launch_deriv_header(h, derivs, s), "derivatives header");
    {
        std::lock_guard<std::mutex> lk(g_deriv_mu);
        g_derivs[derivs] = DerivKey{K, R, p, box};
    }
    return NF_OK;
}

namespace {

// A validated far-field call: its binning plan and the layouts of the
// derivatives buffer and of the workspace.
struct FarCall {
    Plan pl;
    FarLayout F;
    DerivLayout L;
};

int far_prepare(const float* pos, int64_t N, double box, int K, int R, int p, const void* derivs,
                size_t derivs_bytes, void* ws, size_t ws_bytes, FarCall* fc)
{
    int rc = far_validate(K, R, p, box);
    if (rc) return rc;
    if (!pos || !derivs) return fail(NF_ERR_ARG, "null pointer argument");
    fc->L = deriv_layout(K, p);
    if (derivs_bytes < fc->L.total)
        return fail(NF_ERR_ARG, "derivs too small for K = %d, p = %d: %zu bytes given, %zu needed", K, p,
                    derivs_bytes, fc->L.total);
    {
        std::lock_guard<std::mutex> lk(g_deriv_mu);
        auto it = g_derivs.find(derivs);
        if (it != g_derivs.end()) {
            const DerivKey& k = it->second;
            if (k.K != K || k.R != R || k.p != p || k.box != box)
                return fail(NF_ERR_ARG, "derivs were made for K = %d, R = %d, p = %d, box = %g", k.K, k.R, k.p, k.box);
        }
    }
    nf_box b = one_box(N, box, K, 0, 0.0);
    rc = make_plan(&b, 1, false, 32, &fc->pl);
    if (rc) return rc;
    std::vector<size_t> far_guards;
    fc->F = far_layout(fc->pl, K, p, &far_guards);
    fc->pl.guards.insert(fc->pl.guards.end(), far_guards.begin(), far_guards.end());
    rc = check_ws(fc->pl, ws, ws_bytes);
    if (rc) return rc;
    if (ws_bytes < fc->F.total)
        return fail(NF_ERR_WORKSPACE, "far workspace too small: %zu bytes given, %zu needed", ws_bytes, fc->F.total);
    return NF_OK;
}

// Binning, multipoles, convolution, Taylor forces (profile marks when `profile`).
// With binned != nullptr the particles are already binned on this grid (the
// cell offsets and sorted offsets of a near-field call on the same positions)
// and the far call reuses them.
struct Binned {
    const int32_t* off;
    const float4* rel;
    const int32_t* keys;  // cell id of every sorted slot
};

int run_far(const FarCall& fc, const float* pos, int64_t N, double box, int K, int p, const void* derivs,
            double* acc_far, float* acc_add, double* taylors, void* ws, cudaStream_t s, bool profile,
            const Binned* binned = nullptr)
{
    const Plan& pl = fc.pl;
    const FarLayout& F = fc.F;
    const DerivLayout& L = fc.L;
    auto mark = [&](int i) { return profile ? prof_mark(i, s) : cudaSuccess; };
    const int32_t* off = binned ? binned->off : at<int32_t>(ws, pl.o_off);
    const float4* rel = binned ? binned->rel : at<float4>(ws, pl.o_rel);
    const int32_t* keys = binned ? binned->keys : at<int32_t>(ws, pl.o_keys_a);  // sorted cell ids
    NF_CUDA(mark(0), "profile");
    if (!binned) {
        int rc = run_binning(pl, pos, ws, at<int32_t>(ws, pl.o_off), at<float4>(ws, pl.o_rel),
                             at<int32_t>(ws, pl.o_perm), s);
        if (rc) return rc;
    } else {
        int rc = init_ws(pl, ws, s);  // status header and guards of the far workspace
        if (rc) return rc;
    }
    NF_CUDA(mark(1), "profile");
    const int C = (int)pl.C;
    double* M = at<double>(ws, F.o_M);
    double2* Mh = at<double2>(ws, F.o_Mh);
    double2* Th = at<double2>(ws, F.o_Th);
    // cell units throughout: displacements / w (the stored offsets), T'^n = T^n w^{|n|}
    const bool dfl = g_far_arith.load() == NF_FAR_DOUBLE_FLOAT;
    // reduced basis: fold the multipoles, convolve (p+1)^2 fields, rebuild the complete Taylors
    const double w = box / K, V = box * box * box;
    double* Mr = at<double>(ws, F.o_Mr);
    double* s002 = at<double>(ws, F.o_s002);
    char* dv = static_cast<char*>(const_cast<void*>(derivs));
    auto dat = [&](size_t off) { return static_cast<void*>(dv + off); };
    const int* rseg = static_cast<const int*>(dat(L.o_rseg));
    const int* rk = static_cast<const int*>(dat(L.o_rk));
    const double* rcoef = static_cast<const double*>(dat(L.o_rcoef));
    const int i002 = p >= 2 ? 2 : -1;  // (0,0,2): the third term of the complete basis (a, then b, then c)
    // double-float mode: the transforms and the k-space product in double-float too
    const bool dft = dfl;
    if (dfl) {
        // the fold runs inside the multipole kernel; each cell's (0,0,2) term is kept for its sum
        double* m002 = at<double>(ws, F.o_m002);
        NF_CUDA(launch_multipoles_red_df(off, rel, C, p, rseg, rk, rcoef, L.nnz, Mr, dft ? (void*)Mr : nullptr,
                                         m002, s),
                "multipoles (double-float)");
        NF_CUDA(mark(2), "profile");
        if (i002 >= 0) NF_CUDA(launch_far_sum_term(m002, C, 1, 0, s002, s), "sum of the (0,0,2) multipoles");
    } else {
        NF_CUDA(launch_multipoles(off, rel, C, 1.0, p, M, s), "multipoles");
        NF_CUDA(mark(2), "profile");
        NF_CUDA(launch_far_reduce(M, C, L.nt, L.nr, rseg, rk, rcoef, Mr, s), "multipole fold");
        if (i002 >= 0) NF_CUDA(launch_far_sum_term(M, C, L.nt, i002, s002, s), "sum of the (0,0,2) multipoles");
    }
    if (dft) {
        const void* tw = dat(L.o_tw);
        NF_CUDA(launch_far_fft_df(K, L.nr, true, Mr, Mh, nullptr, tw, s), "multipoles (forward transform)");
        NF_CUDA(launch_far_contract_df(K, L.nr, static_cast<const int*>(dat(L.o_seg)),
                                       static_cast<const FarPair*>(dat(L.o_pairs)), dat(L.o_pcdf), dat(L.o_drdf), Mh,
                                       Th, s),
                "convolution");
        NF_CUDA(launch_far_fft_df(K, L.nr, false, nullptr, Th, Mr, tw, s), "Taylors (inverse transform)");
    } else {
        const double2* tw64 = static_cast<const double2*>(dat(L.o_tw64));
        NF_CUDA(launch_far_fft64(K, L.nr, true, Mr, Mh, nullptr, tw64, s), "multipoles (forward transform)");
        NF_CUDA(launch_far_contract(K, L.nr, static_cast<const int*>(dat(L.o_seg)),
                                    static_cast<const FarPair*>(dat(L.o_pairs)),
                                    static_cast<const double*>(dat(L.o_dh)), Mh, Th, s),
                "convolution");
        NF_CUDA(launch_far_fft64(K, L.nr, false, nullptr, Th, Mr, tw64, s), "Taylors (inverse transform)");
    }
    double* T = M;  // the complete multipoles are no longer needed: the rebuilt Taylors go there
    const bool pairs_needed = dfl && (acc_far || acc_add);
    NF_CUDA(launch_far_rebuild(Mr, dft, C, p, L.nt, L.nr, static_cast<const int4*>(dat(L.o_ops)),
                               static_cast<const double2*>(dat(L.o_opf)), i002,
                               4.0 * 3.14159265358979323846 * (double)N * w * w / V,
                               2.0 * 3.14159265358979323846 * w * w / V, i002 >= 0 ? s002 : nullptr,
                               (taylors || !pairs_needed) ? T : nullptr, pairs_needed ? at<void>(ws, F.o_Tdf) : nullptr,
                               s),
            "Taylors (rebuild)");
    NF_CUDA(mark(3), "profile");
    const double scale = 1.0 / ((double)N * (box / K));  // m / w: cell-unit gradient to box units
    if ((acc_far || acc_add) && dfl)
        NF_CUDA(launch_taylor_forces_df(p, keys, rel, at<void>(ws, F.o_Tdf), (int)N, C, scale, acc_far, acc_add, s),
                "Taylor forces (double-float)");
    else if (acc_far || acc_add)
        NF_CUDA(launch_taylor_forces(p, off, rel, T, (int)N, C, 1.0, scale, acc_far, acc_add, s), "Taylor forces");
    NF_CUDA(mark(4), "profile");
    if (profile && g_profile_on) ++g_prof_count;
    if (taylors) NF_CUDA(launch_unscale_taylors(T, C, p, box / K, taylors, s), "Taylors (box units)");
    return NF_OK;
}

}  // namespace

int nf_far_forces(const float* pos, int64_t N, double box, int K, int R, int p, const void* derivs,
                  size_t derivs_bytes, double* acc_far, float* acc_add, double* taylors, void* ws, size_t ws_bytes,
                  void* stream)
{
    g_last_error.clear();
    FarCall fc;
    int rc = far_prepare(pos, N, box, K, R, p, derivs, derivs_bytes, ws, ws_bytes, &fc);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = run_far(fc, pos, N, box, K, p, derivs, acc_far, acc_add, taylors, ws, s, true);
    if (rc) return rc;
    return finish_call(ws, s);
}

int nf_forces_total(const float* pos, int64_t N, double box, int K, int R, double eps, int p, const void* derivs,
                    size_t derivs_bytes, float* acc, void* ws, size_t ws_bytes, void* ws_far, size_t ws_far_bytes,
                    void* stream)
{
    g_last_error.clear();
    nf_box b = one_box(N, box, K, R, eps);
    ForceTuning t;
    int rc = check_tuning(nullptr, &t);
    if (rc) return rc;
    Plan pn;
    rc = make_plan(&b, 1, true, 32 * t.sinks_per_lane, &pn);
    if (rc) return rc;
    if (!pos || !acc) return fail(NF_ERR_ARG, "null pointer argument");
    rc = check_ws(pn, ws, ws_bytes);
    if (rc) return rc;
    FarCall fc;
    rc = far_prepare(pos, N, box, K, R, p, derivs, derivs_bytes, ws_far, ws_far_bytes, &fc);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = run_forces(pn, false, t, pos, nullptr, acc, nullptr, nullptr, ws, s);
    if (rc) return rc;
    const Binned bn{at<int32_t>(ws, pn.o_off), at<float4>(ws, pn.o_rel), at<int32_t>(ws, pn.o_keys_a)};
    rc = run_far(fc, pos, N, box, K, p, derivs, nullptr, acc, nullptr, ws_far, s, false, &bn);
    if (rc) return rc;
    rc = finish_call(ws_far, s);
    if (rc) return rc;
    return finish_call(ws, s);
}

int nf_kdk_step_far(float* pos, float* vel, float* acc, int64_t N, double box, int K, int R, double eps, int p,
                    const void* derivs, size_t derivs_bytes, double* dt, const nf_step_params* prm, void* ws,
                    size_t ws_bytes, void* ws_far, size_t ws_far_bytes, void* stream)
{
    g_last_error.clear();
    nf_box b = one_box(N, box, K, R, eps);
    ForceTuning t;
    int rc = check_tuning(nullptr, &t);
    if (rc) return rc;
    Plan pn;
    rc = make_plan(&b, 1, true, 32 * t.sinks_per_lane, &pn);
    if (rc) return rc;
    if (!pos || !vel || !acc || !dt) return fail(NF_ERR_ARG, "null pointer argument");
    if (prm && (!(prm->eta_acc > 0.0) || !(prm->hubble >= 0.0) || (prm->hubble > 0.0 && !(prm->eta_h > 0.0))))
        return fail(NF_ERR_ARG, "step parameters need eta_acc > 0, hubble >= 0 and eta_h > 0 when hubble > 0");
    rc = check_ws(pn, ws, ws_bytes);
    if (rc) return rc;
    FarCall fc;
    rc = far_prepare(pos, N, box, K, R, p, derivs, derivs_bytes, ws_far, ws_far_bytes, &fc);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    NF_CUDA(launch_kick(vel, acc, (int)N, dt, 0.5, s), "kick");
    NF_CUDA(launch_drift(pos, vel, (int)N, dt, (float)box, s), "drift");
    rc = run_forces(pn, false, t, pos, nullptr, acc, nullptr, nullptr, ws, s);
    if (rc) return rc;
    const Binned bn{at<int32_t>(ws, pn.o_off), at<float4>(ws, pn.o_rel), at<int32_t>(ws, pn.o_keys_a)};
    rc = run_far(fc, pos, N, box, K, p, derivs, nullptr, acc, nullptr, ws_far, s, false, &bn);
    if (rc) return rc;
    NF_CUDA(launch_kick(vel, acc, (int)N, dt, 0.5, s), "kick");
    if (prm)
        NF_CUDA(launch_timestep(at<int32_t>(ws, pn.o_off), at<int32_t>(ws, pn.o_perm), vel, acc, (int)pn.C,
                                (long long)N, prm->eta_acc, prm->eta_h, prm->hubble, at<StepScratch>(ws, pn.o_step),
                                dt, s),
                "time step");
    rc = finish_call(ws_far, s);
    if (rc) return rc;
    return finish_call(ws, s);
}

int nf_set_density_mode(int mode)
{
    g_last_error.clear();
    if (mode < 0 || mode > 2) return fail(NF_ERR_ARG, "density mode %d is not 0 (auto), 1 (fused) or 2 (deferred)", mode);
    g_dens_mode = mode;
    return NF_OK;
}

int nf_get_density_mode(void) { return g_dens_mode; }

int nf_set_debug(int on)
{
    g_debug = on != 0;
    return NF_OK;
}

int nf_debug_check(void* ws, void* stream)
{
    g_last_error.clear();
    if (!ws) return fail(NF_ERR_WORKSPACE, "workspace is NULL");
    if (!g_debug) return fail(NF_ERR_ARG, "debug mode is off: the workspace has no guard blocks");
    return finish_call(ws, static_cast<cudaStream_t>(stream));
}

int nf_status_read(void* ws, void* stream)
{
    g_last_error.clear();
    if (!ws) return fail(NF_ERR_WORKSPACE, "workspace is NULL");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "status sync");
    int bits = 0;
    e = cudaMemcpy(&bits, ws, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (bits & (1 << NF_ERR_NONFINITE)) return fail(NF_ERR_NONFINITE, "non-finite coordinates in the input");
    if (bits & (1 << NF_ERR_TIMEOUT)) return fail(NF_ERR_TIMEOUT, "a device-side wait timed out");
    if (bits & (1 << NF_ERR_CORRUPT)) return fail(NF_ERR_CORRUPT, "a workspace guard block was overwritten");
    return NF_OK;
}

int nf_profile_enable(int on)
{
    g_profile_on = on != 0;
    g_prof_count = 0;
    return NF_OK;
}

namespace {

// the four stage times of a profiled call, `back` calls ago
int profile_stages(int back, float ms[4])
{
    if (back < 0 || back >= NF_PROFILE_RING || back >= g_prof_count)
        return fail(NF_ERR_ARG, "no profiled call %d back (%lld recorded)", back, g_prof_count);
    cudaEvent_t* ev = g_ev[(g_prof_count - 1 - back) % NF_PROFILE_RING];
    cudaError_t e = cudaEventSynchronize(ev[4]);
    if (e != cudaSuccess) return cuda_fail(e, "profile sync");
    for (int i = 0; i < 4; ++i) {
        e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "profile elapsed");
    }
    return NF_OK;
}

}  // namespace

int nf_far_profile_read(int back, nf_far_profile* out)
{
    g_last_error.clear();
    if (!out) return fail(NF_ERR_ARG, "null pointer argument");
    float ms[4];
    const int rc = profile_stages(back, ms);
    if (rc) return rc;
    out->bin_ms = ms[0];
    out->multipoles_ms = ms[1];
    out->convolution_ms = ms[2];
    out->taylor_ms = ms[3];
    out->total_ms = (double)ms[0] + ms[1] + ms[2] + ms[3];
    return NF_OK;
}

int nf_profile_read(int back, nf_profile* out)
{
    g_last_error.clear();
    if (!out) return fail(NF_ERR_ARG, "null pointer argument");
    float ms[4];
    const int rc = profile_stages(back, ms);
    if (rc) return rc;
    out->bin_ms = ms[0];
    out->worklist_ms = ms[1];
    out->pair_ms = ms[2];
    out->combine_ms = ms[3];
    out->total_ms = (double)ms[0] + ms[1] + ms[2] + ms[3];
    return NF_OK;
}

int64_t nf_kernel_launches(void) { return (int64_t)g_launches.load(); }

int nf_stage_stats_read(void* ws, int64_t* out, void* stream)
{
    g_last_error.clear();
    if (!ws || !out) return fail(NF_ERR_ARG, "null pointer argument");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stage stats sync");
    WsHeader h;
    e = cudaMemcpy(&h, ws, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stage stats read");
    out[0] = (int64_t)h.stages;
    out[1] = (int64_t)h.stages_exact;
    out[2] = (int64_t)h.stages_rerun;
    return NF_OK;
}

int nf_stats_read(void* ws, int64_t* out, void* stream)
{
    g_last_error.clear();
    if (!ws || !out) return fail(NF_ERR_ARG, "null pointer argument");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stats sync");
    WsHeader h;
    e = cudaMemcpy(&h, ws, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stats read");
    out[0] = (int64_t)h.pairs;
    out[1] = h.n_items;
    out[2] = h.max_occ;
    out[3] = (int64_t)h.lane_pairs;
    return NF_OK;
}

}  // extern "C"
