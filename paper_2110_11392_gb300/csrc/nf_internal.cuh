// Internal declarations of libnf (not part of the C ABI).
//
// Data layout in device memory (all regions caller-owned, carved out of the
// workspace by nf_api.cu):
//   keys a/b    int32 [N]       cell ids between the sort's passes (a: sorted at the end)
//   rel scratch float4 [N]      offsets between the sort's passes
//   sort ctl    tickets, digit histograms, look-back status words of the sort
//   cell_off    int32 [C+1]     first sorted slot of every global cell
//   rel         float4 [N]      sorted cell-centred offsets, .w = index bits
//   perm        int32 [N]       sorted slot -> particle (global index)
//   items       int4 [<= M]     work items: (global centre cell, chunk, box, -)
//   partial     float4 [N][2R+1]  per-pencil partial sums (ax, ay, az, density),
//                                 one row per particle in original order
// A "global cell" numbers the cells of all boxes of a batch back to back:
// box b owns cells [cell_base_b, cell_base_b + K_b^3).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <vector>
#include <stdint.h>

#include "../../include/nf.h"

namespace nf {

// Per-box constants in device memory.  Lengths in cell units unless noted.
struct BoxDev {
    int K;
    int R;
    int cell_base;   // first global cell of this box
    int part_base;   // first particle (row of pos_cat) of this box
    int N;
    int chunk_base;  // first combine chunk of this box
    double kl;       // K / box, multiplies a box-unit coordinate into cell units
    double scale_acc;   // m / w^2: cell-unit pair sums -> box-unit acceleration
    double scale_grad;  // m / w^3: cell-unit Jacobian sums -> box-unit gradient
    // Eq. (spline) in cell units: f(r) = min(c0 + r^2 (c2 + c1 / r), 1 / r^3)
    float c0, c1, c2;
    float eps2;      // eps_s^2 (cell units^2)
    // f'(r)/r inside the softening: e1 + e0 / r
    float e0, e1;
    // K / box = kl_mant * 2^kl_exp with an odd kl_mant < 2^29, or kl_mant = 0
    // when no such short form exists (then the shift stays in FP64)
    int kl_mant, kl_exp;
    // top-hat density estimate (Sec. "Force Kernel"): b^2 and 1/b^2 in cell units
    float dens_b2, dens_inv_b2;
    // K / box when it is a power of two (then x * K / box is exact in FP32), else 0
    float kl_pow2;
    // 1: the top-hat term runs only in the pair-kernel stages where some pair
    // is closer than b (small b); 0: it is fused into every stage that can hold one
    int dens_defer;
};
static_assert(sizeof(BoxDev) % 16 == 0, "BoxDev must stay 16-byte aligned");

// Header at the start of every workspace (256 bytes).
struct WsHeader {
    int status;          // nf_status bits set on the device
    int queue;           // persistent work queue head
    int n_items;         // number of work items
    int max_occ;         // largest cell occupancy
    unsigned long long pairs;       // sum over pencils of n_sink * n_src
    unsigned long long lane_pairs;  // sink lanes issued * n_src
    // debug mode: byte offsets of the guard blocks that follow each workspace region
    int guard_count;
    int pad0;
    long long guard_off[24];
    // pair-kernel stages: all, on the exact path from the start (the item's own
    // cell), and re-run on the exact path after the fast path met r < eps_s
    unsigned long long stages, stages_exact, stages_rerun;
};
static_assert(sizeof(WsHeader) == 256, "header is 256 bytes");

constexpr int kGuardBytes = 256;       // one guard block (debug mode)
constexpr unsigned kGuardWord = 0xA5C3A5C3u;

constexpr int kMaxBoxesPerFill = 32;
struct BoxFill {
    int first;
    int count;
    BoxDev b[kMaxBoxesPerFill];
};

constexpr int kCombineChunk = 4096;  // particles per combine block (never straddles boxes)
constexpr int kBuckets = 64;         // cost buckets of the LPT work order

// Scratch of the time-step reduction (nf_step.cu).
constexpr int kStepBlocks = 256;
struct StepScratch {
    unsigned min_ratio_bits;  // smallest per-cell v_rms / a_max (bits of a positive float)
    unsigned max_a2_bits;     // largest |a|^2 (bits of a positive float)
    unsigned pad[62];
    double v2_block[kStepBlocks];  // per-block FP64 sums of |v|^2
};

// ---- far field (nf_far.cu) ----
constexpr int kMaxFarOrder = 12;  // NF_MAX_FAR_ORDER
constexpr int kMaxFarTerms = (kMaxFarOrder + 3) * (kMaxFarOrder + 2) * (kMaxFarOrder + 1) / 6;
// One (n, k) pair of the Taylor convolution: terms k and j = n + k (the sign
// bit of j set when |n| + |k| is odd), coefficient (-1)^{|k|} / (n! k!).
struct FarPair {
    int k;
    int j;
    double coef;
};
// Header of a derivatives buffer (nf_derivatives): where its parts live and what it was made for.
struct DerivHeader {
    unsigned magic;
    int K, R, p;
    double box, alpha;
    int nimg, hmax, nt, nr;
    long long npairs;
    unsigned long long o_seg, o_pairs, o_dh, total;  // reduced pair segments and pairs, transformed derivatives
    unsigned long long o_rseg, o_rk, o_rcoef, o_ops, o_opf;  // fold and rebuild tables
    long long nnz;
    unsigned long long o_drdf, o_pcdf, o_tw;  // double-float derivatives, pair coefficients, twiddles
    unsigned long long o_tw64;                 // FP64 twiddles
    unsigned long long pad[11];
};
static_assert(sizeof(DerivHeader) == 256, "derivatives header is 256 bytes");
constexpr unsigned kDerivMagic = 0x4E464452u;
cudaError_t launch_deriv_header(const DerivHeader& h, void* dst, cudaStream_t s);
int far_terms_host(int p);
// Host-built tables of the reduced-basis convolution for order p (cell units,
// cell width w): the fold of complete multipoles onto the (p+1)^2 reduced
// ones (entries grouped by reduced term), the reduced (n, k) pairs, and the
// rebuild program of the complete Taylors (one op per complete term, in an
// order where every op's sources come first).
struct FarTables {
    int nr = 0;
    std::vector<int> red_seg, red_k;
    std::vector<double> red_coef;
    std::vector<int> pair_seg;
    std::vector<FarPair> pairs;
    std::vector<float2> pair_cdf;  // the pairs' coefficients as double-float pairs
    std::vector<int4> ops;       // (dst, reduced source or -1, s1, s2)
    std::vector<double2> opf;    // (f1, f2): T[dst] = -f1 T[s1] - f2 T[s2] (+ the constant for (0,0,2))
    int t002 = -1;               // complete index of (0,0,2), or -1 when p < 2
};
FarTables far_tables(int p, double w);
cudaError_t launch_far_reduce(const double* M, int C, int nt, int nr, const int* seg, const int* kidx,
                              const double* coef, double* Mr, cudaStream_t s);
// per-block partial sums over cells of M[c][term] (far_sum_partials() of them)
cudaError_t launch_far_sum_term(const double* M, int C, int nt, int term, double* partial, cudaStream_t s);
int far_sum_partials();
// complete Taylors T [C][nt] (and, with Tdf, their double-float pairs) from the reduced ones
// Tr: FP64, or double-float pairs with df_in
cudaError_t launch_far_rebuild(const void* Tr, bool df_in, int C, int p, int nt, int nr, const int4* ops,
                               const double2* opf, int t002, double lap, double t0_per_s002, const double* partial,
                               double* T, void* Tdf, cudaStream_t s);
// Factors of K in the order the mixed-radix transforms take them (fours, then
// 2, 3, 5, 7, then any larger prime).
struct Radices {
    int n;
    int r[24];
};
Radices far_radices(int K);
// e^{-2 pi i j / K}, j < K, in FP64
std::vector<double2> far_twiddles64(int K);
// FP64 3-D transforms for any K: forward, real cell-major [K^3][nf] -> complex
// term-major [nf][K][K][K/2+1]; inverse (unnormalised) the reverse (spec is
// overwritten); tw = far_twiddles64(K) in device memory
cudaError_t launch_far_fft64(int K, int nf, bool forward, const double* real_in, double2* spec, double* real_out,
                             const double2* tw, cudaStream_t s);
cudaError_t launch_deriv_real(int K, int R, int p, double box, double alpha, int nimg, double* D, cudaStream_t s);
cudaError_t launch_deriv_recip(int K, int p, double box, double alpha, int hmax, const double2* Dh, double* Dr,
                               cudaStream_t s);
cudaError_t launch_unscale_taylors(const double* Tc, int C, int p, double w, double* T, cudaStream_t s);
// double-float forms of the per-particle kernels (cell units); Tdf holds C * nt pairs of floats (from the rebuild)
// reduced multipoles Mr [C][(p+1)^2] (the fold of the double-float complete ones) and
// each cell's (0,0,2) multipole m002 [C]; rseg/rk/rcoef: the fold table, nnz entries
// (Mrd non-null: the reduced multipoles as double-float pairs there instead of FP64 in Mr)
cudaError_t launch_multipoles_red_df(const int* off, const float4* rel, int C, int p, const int* rseg,
                                     const int* rk, const double* rcoef, long long nnz, double* Mr, void* Mrd,
                                     double* m002, cudaStream_t s);
// Double-float transforms: forward, real cell-major pairs [C][nf] -> spectrum
// [nf][K][K][K/2+1] of float4 {re.h, re.l, im.h, im.l}; inverse (unnormalised),
// spectrum (overwritten) -> real pairs [C][nf].  Radix-4/2 kernels for a
// power-of-two K (4..256, far_df_fft), the mixed-radix ones otherwise.
bool far_df_fft(int K);
std::vector<float4> far_twiddles(int K);  // e^{-2 pi i j/K}, j < K, as double-float pairs
cudaError_t launch_far_fft_df(int K, int nf, bool forward, const void* real_in, void* spec, void* real_out,
                              const void* tw, cudaStream_t s);
// the k-space product on double-float spectra (pcoef: the pairs' coefficients as float2 pairs)
cudaError_t launch_far_contract_df(int K, int nout, const int* seg, const FarPair* pairs, const void* pcoef,
                                   const void* Dr, const void* Mh, void* Th, cudaStream_t s);
cudaError_t launch_to_df(const double* src, long long n, void* dst, cudaStream_t s);
// cell: the cell id of every sorted slot (the binning's sorted keys)
cudaError_t launch_taylor_forces_df(int p, const int* cell, const float4* rel, const void* Tdf, int N, int C,
                                    double scale, double* acc_far, float* acc_add, cudaStream_t s);
// Th[n][q] for nout output fields (the reduced Taylors) from the pair table
cudaError_t launch_far_contract(int K, int nout, const int* seg, const FarPair* pairs, const double* Dr,
                                const double2* Mh, double2* Th, cudaStream_t s);
cudaError_t launch_taylor_forces(int p, const int* off, const float4* rel, const double* T, int N, int C, double w,
                                 double mass, double* acc_far, float* acc_add, cudaStream_t s);

// Counts kernel launches (all translation units).
void count_launches(int n);
// Sets the dynamic shared-memory limit of a kernel once per (device, size).
cudaError_t ensure_smem(const void* fn, int bytes, bool max_carveout = false);

// ---- launch wrappers (nf_bin.cu) ----
cudaError_t launch_fill_boxes(const BoxFill& f, BoxDev* boxes, cudaStream_t s);
// Stable LSD sort of (cell id, particle): digits of at most kSortMaxBits bits,
// one k_sort_pass launch per digit over tiles of kSortTile particles.
constexpr int kSortMaxBits = 9;
constexpr int kSortMaxBins = 1 << kSortMaxBits;
constexpr int kSortMaxPasses = 4;  // cell ids below 2^31 need at most 4 passes of <= 9 bits
constexpr int kSortTile = 2048;
constexpr int kSortWarps = 8;
struct SortPlan {
    int passes;
    int shift[kSortMaxPasses];
    int bits[kSortMaxPasses];
    int tiles;
};
SortPlan sort_plan(int64_t N, int64_t C);
// bytes of the sort's control region (tickets, digit histograms, look-back status words)
size_t sort_ctl_bytes(const SortPlan& p);
// Bins N particles of the boxes: rel [N] (sorted cell-centred offsets, .w =
// index bits), perm [N], cell_off [C+1].  rel_scratch [N], key_a [N], key_b [N]
// and ctl (sort_ctl_bytes) are workspace; key_a ends with the sorted cell ids.
cudaError_t run_sort(const SortPlan& p, const float* pos, int N, int C, const BoxDev* boxes, int nboxes,
                     void* ctl, float4* rel_scratch, int* key_a, int* key_b, float4* rel, int* perm, int* cell_off,
                     WsHeader* hdr, cudaStream_t s);

// ---- work list, force, adjoint, combine (nf_force.cu) ----
struct ForceTuning {
    int sinks_per_lane;
    int stage;
    int warps_per_block;
    int blocks_per_sm;
};

cudaError_t launch_pencils(const BoxDev* boxes, int nboxes, int Ctot, const int* cell_off,
                           int chunk, int stage, int* chunks, unsigned* bucket_count,
                           unsigned char* bucket_of, WsHeader* hdr, cudaStream_t s);
cudaError_t launch_items(const BoxDev* boxes, int nboxes, int Ctot, const int* chunks,
                         const unsigned char* bucket_of, unsigned* bucket_count,
                         int4* items, WsHeader* hdr, cudaStream_t s);
cudaError_t launch_gather_g(const float* g, const int* perm, int Ntot, float4* gs,
                            cudaStream_t s);
cudaError_t launch_force(bool adjoint, bool density, const ForceTuning& t, const BoxDev* boxes,
                         const int* cell_off, const float4* rel, const float4* gs,
                         const int4* items, WsHeader* hdr, float4* partial, int pstride,
                         int max_nseg, cudaStream_t s);
// partial rows of pstride float4 (2 max R + 1) per particle, original order
cudaError_t launch_combine(bool adjoint, const BoxDev* boxes, int nboxes, int nchunks,
                           const float4* partial, int pstride, float* out,
                           float* rho, double* chunk_sums, cudaStream_t s);
cudaError_t launch_net(const BoxDev* boxes, int nboxes, const double* chunk_sums,
                       double* net, cudaStream_t s);
bool force_tuning_supported(const ForceTuning& t);

// ---- cell multipoles (nf_multipole.cu) ----
int multipole_terms(int p);
cudaError_t launch_multipoles(const int* off, const float4* rel, int C, double w, int p, double* M, cudaStream_t s);

// ---- time stepping (nf_step.cu) ----
cudaError_t launch_kick(float* vel, const float* acc, int N, const double* dt, double factor, cudaStream_t s);
cudaError_t launch_drift(float* pos, const float* vel, int N, const double* dt, float box, cudaStream_t s);
cudaError_t launch_timestep(const int* off, const int* perm, const float* vel, const float* acc, int C, long long N,
                            double eta_acc, double eta_h, double hubble, StepScratch* st, double* dt,
                            cudaStream_t s);
int force_blocks_per_sm(bool adjoint, bool density, const ForceTuning& t, int max_nseg);

}  // namespace nf
