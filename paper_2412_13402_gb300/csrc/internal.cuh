// internal.cuh -- declarations shared by the translation units of librtbte.
//
// Data layout in HBM (one context, several independent instances):
//   state y (FP64, caller-owned)   [inst0: f (n_c) | N (nmodes*N_q)] [inst1: ...] ...
//   population copies (compute precision R, written once per RHS by the stage kernels):
//     popf  electron f per instance, padded to a multiple of 4 elements
//     popN  phonon N per instance as [mode][q] with the q stride padded to a multiple of 4,
//           so the slice of one mode is a 16-byte aligned block for staging
//     popP  N on the ph-ph sub-lattice (compact index a = nu*N_q,pp + qs_lin), padded
//   channel lists (per instance, per part): uint32 packed index + weight (R), CSR offsets
//     e-ph  segments (nu, d, proc) -> idx = s | q << s_bits     (q = phonon q_lin of mode nu)
//     ph-e  segments p             -> idx = d | s << s_bits
//     ph-ph segments (a, proc)     -> idx = b | c << pp_bits
//     every segment is padded with zero-weight entries to a multiple of 4 entries so that a
//     warp reads 4 entries per lane with one 16-byte load.
//   work items: <= 512 entries of one segment, processed by one warp, which writes one
//   compensated partial sum (hi, lo); rows combine their items' partials in item order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "rtbte.h"

namespace rtbte {

constexpr int kItemEntries = 512;  // 32 lanes x 4 vectors x 4 entries
constexpr int kSegPad = 4;
constexpr int kRhsThreads = 512;      // collision kernel, threads per SM: two register buffers of entries per warp
constexpr int kRhsThreadsDeep = 768;  // FP32 single-buffer form: 24 warps per SM at 80 registers
constexpr int kMaxModes = 16;
constexpr int kMaxStages = 5;
constexpr int kWrmsBlocks = 512;
constexpr int kWrmsChunks = 128;  // per-instance blocks of the WRMS reduction before the controller
constexpr int kMaxBatch = 1024;  // instances per context (shared-memory tables of the batched kernels)
constexpr int kLoopCap = 64;     // attempts per launch of an attempt-loop graph (default)

enum { PART_EPH = 0, PART_PHE = 1, PART_PP = 2 };
// Lanes working on one item are chosen per staging group (Group::lanes_log2): 4, 8, 16 or 32 lanes,
// items of at most 16 x lanes entries, so that groups of short segments pack several items into
// one warp while groups of long segments keep whole-warp items.


// A work item as stored (16 B): up to kItemEntries entries of one destination segment.
struct __align__(16) ItemRec {
    unsigned int begin_lo;   // first entry (bits 0-31), relative to the group's entry arrays
    unsigned int slot;       // index of the item's partial: the items of one row have consecutive
                             // slots, in the order the row adds them
    int dest;                // instance-local destination (electron d, phonon p, sub-lattice a)
    unsigned short len;      // entries (multiple of 4, <= kItemEntries)
    unsigned char proc;      // 0 emission, 1 absorption
    unsigned char begin_hi;  // first entry, bits 32-39
};

// A work item as the collision kernel uses it.
struct Item {
    long long begin;
    unsigned int slot;
    int dest;
    unsigned short len;
    unsigned char proc;
};

// Consecutive items that share one shared-memory staging of populations.
struct __align__(16) Group {
    const uint32_t *idx;  // entry arrays of this instance and part
    const void *W;
    int item_begin, item_end;
    int part, inst, nu, s_bits;
    int pp_bits, n_q_pad;
    int lanes_log2, pad_g;       // lanes per item = 1 << lanes_log2 (2, 3, 4 or 5)
    int stage0_len, stage1_len;  // staged element counts (multiples of 4)
    int stage1_q0, pad_s;        // e-ph: first q of the staged block of the mode's N
    long long stage0_src;        // popf (e-ph, ph-e) or popP (ph-ph) offset of the staged block
    long long stage1_src;        // popN offset of the staged mode slice (e-ph)
    long long f_inst, N_inst, P_inst;  // instance offsets in popf / popN / popP
};

// Per-instance layout used by the row kernels.
struct __align__(16) InstDev {
    long long y_off;
    int n_c, n_ph, M, nmodes;
    int N_q, N_q_pad;
    long long f_off, N_off, P_off;  // offsets in popf / popN / popP
    long long compact_base;         // sub-lattice index of each phonon (-1: none): [n_ph]
};

// Device-side controller state of the adaptive integrators (one per instance).
struct __align__(16) Ctl {
    double t, t_out, h, h_try;
    double eps, eps1, eps2, h_last;
    double h0tmp, span_t0, pad_d0, pad_d1;
    long long steps, attempts, fails, rhs;
    long long max_steps, steps_base, range_viol, pad_l1;  // range_viol: out-of-range rows in accepted steps
    int first, nef, done, status;
    int cur, last, fixed, pad_i0;
};

// Launch parameters of the collision kernel for one parts mask.
struct LaunchTuning {
    int w = 320;                     // work-split weight of an item beyond its entries
    int pf = 3;                      // L2 prefetch distance in items of a warp's sequence (0: off)
    double sf = 1.0;                 // share of the weight split statically (rest: dynamic chunks)
    double ps[3] = {1.0, 1.0, 1.0};  // relative cost of an entry of each part
    bool deep = false;               // FP32: the single-buffer form at 24 warps per SM
};

struct CtlParams {  // constants of one integration (captured into graphs by value)
    double rtol, atol_c, atol_ph;
    double a1, a2, a3, safety, growth, growth_first, etamxf, etamin, hmin, hmax;
    int p, pid_sign_mode, small_nef, max_nef;
};

struct Tableau {
    int S, p, has_emb, pad;
    double A[kMaxStages][kMaxStages];
    double b[kMaxStages], bt[kMaxStages], c[kMaxStages];
};

// ---- small device helpers -------------------------------------------------
__host__ __device__ inline int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}
__host__ __device__ inline int min_image(int d, int n) {
    d = wrapi(d, n);
    return d > n / 2 ? d - n : d;
}
// SplitMix64 output function (Steele, Lea & Flood 2014), used as a keyed hash.
__host__ __device__ inline unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
inline int bits_for(long long n) {  // bits needed for indices 0..n-1
    int b = 1;
    while ((1LL << b) < n) ++b;
    return b;
}
inline long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// The dynamic shared-memory limit is an attribute of the kernel function, shared by every
// context (and surrogate) of the process: it is set to the device's opt-in maximum less the
// kernel's static shared memory, so that no context lowers it below another's launches.
inline cudaError_t allow_max_dynamic_smem(const void *f) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   optin - (int)fa.sharedSizeBytes);
    return e;
}

// ---- device buffer ----------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// Builder input tables of one instance on the device.
struct BuildTables {
    const int4 *ek;                       // (kx, ky, kz, band) per electron state
    const double *eps;                    // [n_c]
    const unsigned long long *eid, *eid_inv;  // electron grid ids of k and -k
    const double *omega;                  // [nmodes*N_q]
    const int *kmap;                      // [nbands*N_k] state index or -1
    const double *lut;                    // [2^lut_bits]
    const double *g2;                     // [nmodes]
    const int *pp_full, *pp_full_inv;     // [M] full phonon index of a and of its -q image
    int n_c, nbands, nmodes, fold, lut_bits;
    int nk[3], nq[3], nqs[3];
    long long N_k, N_q, N_ph, M, N_qs;
    int s_bits, q_bits, pp_bits;
    int eph_nqb, eph_qblk;  // e-ph q-blocks per mode, q points per block
    long long row_lo, row_hi;  // fill passes store only destinations whose state row is in [row_lo, row_hi)
    double cut_eph, cut_pp, sigma_eph, sigma_pp, omega_cut;
    double pref_eph, pref_phe, pref_pp;  // 2pi/(hbar N_q), 4pi/(hbar N_k), 36pi/(hbar N_q,pp)
    double v3;
    unsigned long long g2_seed, v3_seed;
};

struct InstHost {
    rtbte_instance_desc d{};
    std::vector<int32_t> e_band, e_k;
    std::vector<double> e_eps, ph_omega, lut, g2_coef;
    long long N_k = 0, N_q = 0, n_ph = 0, M = 0, N_qs = 0;
    int nqs[3] = {1, 1, 1};
    int N_q_pad = 0, n_c_pad = 0, M_pad = 0;
    int s_bits = 0, q_bits = 0, pp_bits = 0;
    int eph_nqb = 1, eph_qblk = 0;  // e-ph q-blocks per mode and their size in q points (multiple of 4)
    std::vector<int32_t> pp_full, pp_full_inv, compact;
    // builder tables (device), kept for rebuilds
    DevBuf t_ek, t_eps, t_eid, t_eidinv, t_omega, t_kmap, t_lut, t_g2, t_ppfull, t_ppinv;
    // channel lists (device)
    DevBuf eph_idx, eph_W, phe_idx, phe_W, pp_idx, pp_W;
    std::vector<long long> eph_off, phe_off, pp_off;  // padded CSR offsets (host copy)
    DevBuf pp_off_dev;                                // device copy of pp_off (made on first use)
    std::vector<long long> eph_cnt, phe_cnt, pp_cnt;  // logical counts per segment (0 outside the row slice)
    // padded segment lengths over EVERY row (row slices included), from which the plan takes each
    // staging group's lanes per item, so that a sliced context cuts its items like a full one
    std::vector<long long> eph_plen, phe_plen, pp_plen;
    long long row_lo = 0, row_hi = 0;  // state-row slice [row_lo, row_hi) of this instance (all rows: 0, n_y)
    bool has_channels = false;
    bool counted = false;  // per-segment counts exist (after any upload mode, RTBTE_CH_COUNT included)
    long long y_off = 0, f_off = 0, N_off = 0, P_off = 0;
};

}  // namespace rtbte

struct rtbte_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int precision = RTBTE_PREC_FP32_COMP;
    size_t real_size = 4;
    double hbar = 6.582119569e-4;
    std::vector<rtbte::InstHost> inst;
    long long n_y = 0;
    long long popf_len = 0, popN_len = 0, popP_len = 0;
    rtbte::DevBuf popf, popN, popP, instdev, compact;
    // execution plan of the RHS
    bool plan_valid = false;
    rtbte::DevBuf items, groups, partials, rowoff, rowmid, cta_tab, gwt, dyn_tab;  // rowoff/rowmid: slots of each row
    int n_rblk = 0;  // several instances: row blocks of the stage kernels (256 rows of one instance each)
    int n_items = 0, n_groups = 0;
    int part_items[3] = {0, 0, 0};
    int part_first[3] = {0, 0, 0};
    int stage_resident = 0;    // stage kernel: blocks resident on the whole GPU at once (its grid)
    int grid = 0, per_sm = 1;  // collision kernel: CTAs per SM (1, 2 or 4; threads = form's threads per SM / per_sm)
    rtbte::LaunchTuning lt[8];  // collision-kernel launch parameters of each parts mask (1..7)
    unsigned lt_tuned = 0;      // masks the autotuner tuned themselves (kept across plans)
    std::vector<unsigned short> item_len_h;  // entries per work item (host copy for re-splitting)
    std::vector<int> group_begin_h;          // first item of each group (host copy)
    rtbte::DevBuf tail_tab, tail_ctr;        // dynamic chunks {first, end, group, 0} per mask; grab/exit counters
    int tail_off[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // chunks of mask m: [tail_off[m-1], tail_off[m])
    size_t smem_bytes = 0;
    bool staged = false;
    bool wide = true;  // every group uses whole-warp items (the kernel variant without sub-warps)
    int num_sms = 0;
    size_t smem_optin = 0;
    // integrator work buffers
    rtbte::DevBuf Y[2], K, Fs, forcing, wrms_part, ctl, ystage, ydstage, range_scratch;  // wrms_part: 2 x n_y squared norms, then per-instance chunk sums
    rtbte::Ctl *ctl_host = nullptr;  // pinned mirror of the per-instance controllers
    rtbte::DevBuf slow_save;          // tolerance-chosen MRI: y_n, the single-step result, error norms
    double h_slow = 0.0;              // tolerance-chosen MRI: slow step proposal after the last call
    int eph_q_blocks = 0;             // requested e-ph q-blocks (0: automatic)
    bool sliced = false;              // the single instance evaluates a row slice only (rtbte_desc)
    std::map<long long, cudaGraphExec_t> graphs;
    std::map<long long, int> graph_launches;  // kernels per attempt of each attempt-loop graph
    bool use_graphs = true;                   // attempts through the device-loop graph (else direct launches)
    rtbte::DevBuf loop_iter;                  // attempts run by the last attempt-loop launch (device)
    int *loop_iter_host = nullptr;            // pinned mirror
    long long launches = 0;
    // surrogate of the slow part used by MRI integrations (not owned)
    rtbte_surrogate *sur = nullptr;
    std::vector<rtbte_surrogate *> surs;  // every live surrogate made on this context
    int sur_period = 10;
    double sur_tol = 1e-2;
    // collision-kernel timing (events recorded around launches outside graphs)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;            // free events
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    std::string err;
};

namespace rtbte {
// builder.cu
int build_channels(rtbte_ctx *ctx, int inst, bool count_only);
int upload_tables(rtbte_ctx *ctx, int inst);
// rhs.cu
int make_plan(rtbte_ctx *ctx);
int launch_prep_from_y(rtbte_ctx *ctx, const double *y, cudaStream_t s);
int launch_rhs_core(rtbte_ctx *ctx, unsigned parts, const Ctl *ctl, cudaStream_t s);
int launch_rows(rtbte_ctx *ctx, unsigned parts, double *out, const double *forcing, cudaStream_t s);
int split_tables(rtbte_ctx *ctx);
int autotune(rtbte_ctx *ctx, unsigned parts, int *chosen);
// integrate.cu
int advance_to(rtbte_ctx *ctx, double t_out, double *y, const rtbte_integ *opt, rtbte_stats *st);
void destroy_graphs(rtbte_ctx *ctx);
int init_stage_grid(rtbte_ctx *ctx);  // resident blocks of the stage kernel (before any capture)
// api.cu
int fail(rtbte_ctx *ctx, int code, const std::string &msg);
int launch_pp_rates(rtbte_ctx *ctx, int inst, double *rates, cudaStream_t s);
// Surrogate slow value (control variate about the last exact reference) at the device state y,
// written to dst [n_y]; and the judge, which compares that value with the exact one and makes
// (y, exact) the new reference (*relerr < 0 when there was no reference yet).
int sur_value(rtbte_ctx *ctx, const double *y, double *dst);
int sur_judge(rtbte_ctx *ctx, const double *y, const double *exact, double *relerr);
void sur_reset(rtbte_ctx *ctx);  // forget the reference (the next judge only sets it)
void sur_orphan(rtbte_ctx *ctx); // the context goes away: its surrogates refuse further work
int cuda_fail(rtbte_ctx *ctx, cudaError_t e, const char *what);
}  // namespace rtbte

#define RT_CUDA(ctx, call)                                         \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return rtbte::cuda_fail(ctx, e_, #call); \
    } while (0)
