/*
 * rtbte.h -- C ABI of the GB300 (sm_103a) library for the coupled electron/phonon
 * real-time Boltzmann equation (rt-BTE) of arXiv 2412.13402.
 *
 * The library evaluates the right-hand side of Eq. bte,
 *     df_{nk}/dt  = I^{e-ph}[f, N]                    (Eq. e-ph, first integral)
 *     dN_{nu q}/dt = I^{ph-e}[f, N] + I^{ph-ph}[N]     (Eq. e-ph second integral, Eq. ph-ph)
 * on the state vector y = [f_{nk}; N_{nu q}] (Eq. state_vec), and advances it with the
 * integrators of Methods B: fixed-step RK4, adaptive explicit RK with an embedded error
 * estimate (Eq. ERK_method), the WRMS norm (Eqs. wrms_norm, wrms_weights), the PID step
 * controller (Eq. pid_controller), and the explicit MRI/MIS method (Eq. mis_coef) with the
 * fast/slow split of Eq. mri_rhs.  The scattering channels are "computed and stored before
 * the real-time simulation" (Results, rt-BTE section); rtbte_upload_channels builds or
 * copies them.
 *
 * Conventions
 *   - Units: energies in eV (phonon tables hold hbar*omega), time in ps, hbar in eV*ps.
 *   - Every call returns RTBTE_OK (0) or a negative RTBTE_E_* code; rtbte_last_error()
 *     gives a one-line message.  No call traps the device or aborts the process.
 *   - Host arrays passed in descriptors are read during the call only (the library keeps
 *     its own copies).  Device arrays (y, ydot) are owned by the caller.
 *   - All GPU work is ordered on the context's stream; the calls return when their work
 *     is enqueued, except where stated (rtbte_advance_to and host-pointer rtbte_rhs
 *     synchronise the stream before returning).
 *   - One context serves one device; it is not thread-safe (one host thread at a time).
 */
#ifndef RTBTE_H
#define RTBTE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTBTE_VERSION 1

/* ---- status codes ------------------------------------------------------- */
#define RTBTE_OK 0
#define RTBTE_E_INVALID_ARG (-1)    /* bad pointer, size or option                       */
#define RTBTE_E_OOM (-2)            /* device or host allocation failed                  */
#define RTBTE_E_CUDA (-3)           /* a CUDA runtime call failed                        */
#define RTBTE_E_TOO_MANY_STEPS (-4) /* max_steps reached before t_out                    */
#define RTBTE_E_STEP_UNDERFLOW (-5) /* step size fell below hmin                         */
#define RTBTE_E_ERR_TEST_FAIL (-6)  /* max_nef consecutive error-test failures           */
#define RTBTE_E_NONFINITE (-7)      /* NaN/Inf in a stage, the solution or the norm      */
#define RTBTE_E_TIMEOUT (-8)        /* a bounded device wait gave up                     */
#define RTBTE_E_STATE (-9)          /* call out of order (e.g. rhs before channels)      */
#define RTBTE_E_UNSUPPORTED (-10)   /* sizes beyond the packed-index formats             */

/* ---- right-hand-side parts (Eq. erk_rhs / Eq. mri_rhs) ------------------- */
#define RTBTE_EPH 1u  /* I^{e-ph}: electron rows                                        */
#define RTBTE_PHE 2u  /* I^{ph-e}: phonon rows fed by e-ph absorption                   */
#define RTBTE_PHPH 4u /* I^{ph-ph}: phonon rows, three-phonon processes                 */
#define RTBTE_FAST (RTBTE_EPH | RTBTE_PHE)
#define RTBTE_SLOW RTBTE_PHPH
#define RTBTE_ALL (RTBTE_EPH | RTBTE_PHE | RTBTE_PHPH)

/* ---- arithmetic of the collision sums ------------------------------------ */
#define RTBTE_PREC_FP32_COMP 0 /* FP32 gathers/products, compensated FP32 sums, FP64 out */
#define RTBTE_PREC_FP64 1      /* FP64 weights, populations, products and sums          */

/* One simulation instance: grids, bands, phonon branches, couplings (Methods A).
 * Electron state s (0..n_c-1) is the s-th kept (band, k) pair in the order the caller
 * lists them; e_k gives its integer grid coordinates on the nk grid.  Phonon state
 * p = nu*N_q + q_lin with q_lin = (qz*nq[1] + qy)*nq[0] + qx.  The phonon wave vector of
 * the e-ph term linking k (destination) to k' (source) is q = T(k' - k): the minimum-image
 * difference on the electron grid (each component in (-nk/2, nk/2]) divided by `fold`
 * with truncation, modulo nq.  ph-ph acts on the phonons whose q coordinates are all
 * multiples of pp_stride (pp_stride = 0: no ph-ph).  Coupling strengths are
 * |g|^2 = g2_coef[nu] * lut[i] and |V3|^2 = v3_coef * lut[i], where i is the top lut_bits
 * bits of h = mix64(key ^ mix64(seed)), mix64 being SplitMix64's output function
 * (z += 0x9E3779B97F4A7C15; z = (z^(z>>30))*0xBF58476D1CE4E5B9; z = (z^(z>>27))*0x94D049BB133111EB;
 * z^(z>>31)).  e-ph key: with u = band*N_k + k_lin for the two electron states and v their
 * images under k -> -k, take the sorted pairs (lo,hi) of u and of v, keep the
 * lexicographically smaller, key = (lo*U + hi)*nmodes + nu, U = nbands*N_k.  ph-ph key:
 * the full phonon indices of the three participants sorted, likewise for their q -> -q
 * images, the smaller triple (t1,t2,t3) gives key = (t1*N_ph + t2)*N_ph + t3.  Both keys,
 * and hence the couplings, are symmetric under exchange of the participants and inversion. */
typedef struct rtbte_instance_desc {
    int32_t dim;       /* 2 or 3                                                   */
    int32_t fold;      /* nk[c] / nq[c] for every used dimension (1 or 2)          */
    int32_t nbands;    /* electron bands                                            */
    int32_t nmodes;    /* phonon branches                                           */
    int32_t nk[3];     /* electron grid (nk[2] = 1 in 2D)                          */
    int32_t nq[3];     /* phonon grid                                               */
    int32_t n_c;       /* kept electron states                                      */
    int32_t pp_stride; /* ph-ph sub-lattice stride (0: no ph-ph)                    */
    int32_t lut_bits;  /* log2 of the coupling look-up table length (1..20)        */
    int32_t reserved0;
    const int32_t *e_band;   /* host [n_c]                                          */
    const int32_t *e_k;      /* host [n_c*3] grid coordinates                        */
    const double *e_eps;     /* host [n_c] band energies, eV                          */
    const double *ph_omega;  /* host [nmodes*N_q] hbar*omega, eV                     */
    const double *lut;       /* host [2^lut_bits] lognormal shape factors            */
    const double *g2_coef;   /* host [nmodes] |g|^2 medians, eV^2                    */
    double v3_coef;          /* |V3|^2 median                                        */
    double sigma_eph;        /* Gaussian broadening of I^{e-ph}, I^{ph-e}, eV        */
    double sigma_pp;         /* Gaussian broadening of I^{ph-ph}, eV                 */
    double omega_cut;        /* phonons with hbar*omega below this are frozen, eV     */
    uint64_t g2_seed, v3_seed;
} rtbte_instance_desc;

typedef struct rtbte_desc {
    int32_t n_instances;  /* independent simulations sharing one state vector (1..1024;
                             the first collision evaluation refuses more than 1024
                             instances or staging groups with UNSUPPORTED)             */
    int32_t precision;    /* RTBTE_PREC_*                                           */
    const rtbte_instance_desc *inst; /* host [n_instances]                           */
    double hbar;          /* eV*ps                                                   */
    void *stream;         /* cudaStream_t used for every launch (NULL: default stream) */
    int32_t device;       /* CUDA device ordinal (must be current for every call)    */
    int32_t eph_q_blocks; /* built e-ph lists of each mode split by phonon wavevector into
                             this many contiguous q-blocks, so that the populations a block
                             reads (f and that block of the mode's N) fit in shared memory:
                             0 = automatic (1 when f and the whole mode's N fit, else the
                             fewest equal blocks that fit); prebuilt lists always use 1.
                             Segment order of built e-ph lists: (mode, block, electron,
                             process), sources ascending within a segment               */
    /* Row slice (the destination-row split of one instance over several processes or GPUs;
     * the sums over k and q of Eq. e-ph and Eq. ph-ph are independent per destination row).
     * Single-instance contexts only: with row_end > row_begin the context evaluates only the
     * state rows [row_begin, row_end) of y (electron rows 0..n_c-1 first, then phonon rows
     * n_c + p): channel lists are stored for those destinations alone, rtbte_rhs writes 0 on
     * every other row, and each owned row gets the same bits as in an unsliced context (the
     * builder counts every row so that the work items are cut alike).  The caller gathers the
     * slices (e.g. an all-gather, or a sum all-reduce since other rows are 0).
     * rtbte_advance_to refuses a sliced context (STATE).  0, 0: every row. */
    int64_t row_begin, row_end;
} rtbte_desc;

/* Channel source for rtbte_upload_channels.
 * mode RTBTE_CH_BUILD: the device builder enumerates the channels from the instance
 *   tables (all other fields ignored).
 * mode RTBTE_CH_PREBUILT: host CSR arrays in the library's logical order (no padding):
 *   e-ph  segments g = (nu*n_c + d)*2 + proc (proc 0 emission, 1 absorption), entries
 *         (src electron, full phonon p) sorted by src, weight (2 pi/hbar)(1/N_q)|g|^2 delta;
 *   ph-e  segments p (all nmodes*N_q phonons), entries (dest electron d, source s) sorted
 *         by (d, s), weight (4 pi/hbar)(1/N_k)|g|^2 delta;
 *   ph-ph segments g = a*2 + proc over the M sub-lattice phonons, entries (b, c) sorted by
 *         (b, c); emission lists unordered pairs b <= c with weight doubled for b != c,
 *         absorption weight is 2 (36 pi/hbar)(1/N_q,pp)|V3|^2 delta.
 *   Weights are FP64 on input and stored in the context precision. */
#define RTBTE_CH_BUILD 0
#define RTBTE_CH_PREBUILT 1
#define RTBTE_CH_COUNT 2 /* count every row's channels on the device without storing them (for
                            rtbte_row_entries, e.g. to balance row slices); the instance still has
                            no channels afterwards */
typedef struct rtbte_channels {
    int32_t mode;
    int32_t reserved;
    const int64_t *eph_off; const int32_t *eph_src; const int32_t *eph_ph; const double *eph_W;
    const int64_t *phe_off; const int32_t *phe_dst; const int32_t *phe_src; const double *phe_W;
    const int64_t *pp_off; const int32_t *pp_b; const int32_t *pp_c; const double *pp_W;
} rtbte_channels;

/* Per-instance sizes after channels exist. */
typedef struct rtbte_sizes {
    int64_t n_c, n_ph, n_pp, y_offset, n_y_total;
    int64_t eph_entries, phe_entries, pp_entries;        /* logical entries          */
    int64_t eph_stored, phe_stored, pp_stored;           /* stored, incl. padding    */
    int64_t work_items;                                  /* whole context            */
    int64_t channel_bytes;                               /* device bytes, this inst. */
    int64_t eph_q_blocks;                                /* q-blocks per mode of the stored
                                                            e-ph lists (rtbte_desc)    */
} rtbte_sizes;

/* ---- integrators (Methods B) --------------------------------------------- */
#define RTBTE_RK4 0       /* classical RK4, fixed step h                                 */
#define RTBTE_BS32 1      /* adaptive Bogacki-Shampine 3(2)                              */
#define RTBTE_ZON43 2     /* adaptive Zonneveld 4(3) (ARKODE's default ERK)               */
#define RTBTE_MRI_KW3 3   /* MIS on Knoth-Wolke, fixed slow step h_s, adaptive fast ERK  */
#define RTBTE_SPLIT_RK4 4 /* first-order splitting: RK4 slow step h_s, RK4 fast steps h  */
#define RTBTE_MRI_ADAPT 5 /* MIS on Knoth-Wolke with the slow step chosen from rtol/atol by
                             step doubling (the extension the Discussion names as future
                             work: slow and fast steps both from tolerances), adaptive fast
                             ERK; the learned slow stage is not used by this method      */

typedef struct rtbte_integ {
    int32_t method;        /* RTBTE_RK4 .. RTBTE_MRI_ADAPT                                */
    int32_t fast_method;   /* inner ERK of MRI: RTBTE_ZON43 (default) or RTBTE_BS32      */
    double t0;             /* time of the incoming state y                                */
    double h;              /* RK4 step; SPLIT_RK4 fast step                               */
    double h_s;            /* MRI / SPLIT_RK4 slow step; MRI_ADAPT: first slow step       */
    double rtol, atol_c, atol_ph;   /* Eq. wrms_weights; atol per carrier / phonon row   */
    double h0;             /* first step (<= 0: Hairer-Norsett-Wanner estimate)           */
    double hmin, hmax;     /* 0: unbounded                                                */
    int64_t max_steps;     /* accepted-step limit per call (0: 10^9)                      */
    double a1, a2, a3;     /* PID gains (Eq. pid_controller), p* = method order           */
    int32_t pid_sign_mode; /* 0: eps_k^-a1 eps_{k-1}^+a2 eps_{k-2}^-a3; 1: all negative    */
    int32_t max_nef;       /* consecutive error-test failures allowed (default 7)         */
    double safety, growth, growth_first, etamxf, etamin; /* 0: library defaults          */
    int32_t small_nef;     /* failures before etamxf applies (default 2)                  */
    int32_t chunk;         /* attempts per launch of the device attempt loop (0: 64)      */
    int32_t resume;        /* 1: continue the controller of the previous call (step proposal,
                              error history; no first-step estimate; MRI_ADAPT: also the slow
                              step proposal) -- see rtbte_controller                          */
    int32_t reserved2;
    /* MRI_ADAPT only (not in the paper; 0 selects the library default in brackets).  Each slow
     * attempt from y_n takes one MIS step of H (y_1) and two of H/2 (y_2); the local error of
     * y_2 is (y_1 - y_2) / (2^3 - 1), its WRMS norm eps uses rtol, atol_c, atol_ph and weights
     * from y_n (Eq. wrms_norm, Eq. wrms_weights), the largest eps over instances decides:
     * eps <= 1 accepts y_2, else y_n is restored.  Next H = H * min(fac_max, max(fac_min,
     * safety * eps^(-1/4))), the factor at most 1 after a rejection and on the next attempt. */
    double fast_tol_scale; /* fast ERK runs at rtol, atol_c, atol_ph times this [0.1]         */
    double slow_safety;    /* [0.9]                                                           */
    double slow_fac_min;   /* [0.2]                                                           */
    double slow_fac_max;   /* [5]                                                             */
    int32_t slow_max_fail; /* consecutive rejected slow steps before ERR_TEST_FAIL [7]        */
    int32_t reserved3;
} rtbte_integ;

/* Step-size controller state of one instance (Eq. pid_controller), for checkpointing: save it
 * with the state vector after rtbte_advance_to, restore both into a new context, and a call
 * with opt->resume = 1 continues exactly as the uninterrupted run would. */
typedef struct rtbte_controller {
    double t;          /* time of the state it belongs to                                   */
    double h;          /* next step proposal                                                */
    double eps1, eps2; /* error history eps_{k-1}, eps_{k-2}                                */
    int32_t first;     /* 1 before the first accepted step                                  */
    int32_t nef;       /* consecutive error-test failures                                   */
} rtbte_controller;

typedef struct rtbte_stats {
    int64_t steps, attempts, fails;      /* accepted steps, attempts, error-test fails    */
    int64_t rhs_full, rhs_fast, rhs_slow;/* RHS evaluations by part set                   */
    int64_t slow_steps;                  /* MRI / split slow steps                        */
    double t;                            /* time of the returned y                        */
    double h_last, h_next;               /* last accepted step, next proposal             */
    int32_t status;                      /* same as the return value                      */
    int32_t surrogate_fallbacks;         /* MRI calls that detached the surrogate (0/1)   */
    int64_t slow_exact, slow_surrogate;  /* MRI slow stages: exact / surrogate values     */
    double judge_err_max;                /* largest relative error seen by a judge (or -1)*/
    int64_t range_violations;            /* rows of accepted step states with f outside
                                            [-atol_c, 1+atol_c] or N < -atol_ph           */
    int64_t slow_fails;                  /* MRI_ADAPT: rejected slow attempts             */
    double h_slow_next;                  /* MRI_ADAPT: next slow step proposal            */
} rtbte_stats;

typedef struct rtbte_ctx rtbte_ctx;

/* Fill `d` with defaults (1 instance, FP32_COMP, hbar = 6.582119569e-4 eV*ps, device 0). */
void rtbte_desc_defaults(rtbte_desc *d);
/* Fill `o` with the paper's defaults: PID a1=0.58, a2=0.21, a3=0.1 (Methods B) and ARKODE's
 * documented controller constants for what the paper leaves unstated. */
void rtbte_integ_defaults(rtbte_integ *o);

/* Create a context: copies the instance tables to the device and allocates the state-size
 * work buffers.  Errors: INVALID_ARG (bad desc), OOM, CUDA. */
int rtbte_create(const rtbte_desc *d, rtbte_ctx **out);

/* Build (mode BUILD) or copy (mode PREBUILT) the channel lists of instance `inst`.  Device
 * builder: one-time enumeration of every (destination, source, mode, process) term whose
 * energy mismatch is within 3 sigma and whose phonons are above omega_cut; FP64 filter with
 * IEEE add/sub only, so the lists are bit-identical to any IEEE implementation of the same
 * rule.  Replaces earlier channels of the instance.  Errors: INVALID_ARG, UNSUPPORTED
 * (an index does not fit the packed 32-bit entry format), OOM, CUDA. */
int rtbte_upload_channels(rtbte_ctx *ctx, int inst, const rtbte_channels *ch);

/* ydot = selected parts of the RHS at y (time t is accepted for interface symmetry; the
 * rt-BTE RHS is autonomous).  y and ydot are FP64 [n_y_total] arrays, either both device
 * pointers (stream-ordered, asynchronous) or both host pointers (staged through the
 * context, synchronous).  Rows of parts not selected are written as 0.
 * Errors: STATE (some instance has no channels), INVALID_ARG, CUDA. */
int rtbte_rhs(rtbte_ctx *ctx, double t, const double *y, double *ydot, unsigned parts);

/* Read / write the controller state of instance `inst` (host memory).  get reflects the end
 * of the last rtbte_advance_to (or the last set); set takes effect at the next call with
 * opt->resume = 1.  Errors: INVALID_ARG. */
int rtbte_get_controller(const rtbte_ctx *ctx, int inst, rtbte_controller *out);
int rtbte_set_controller(rtbte_ctx *ctx, int inst, const rtbte_controller *in);

/* Linearised ph-ph scattering rates (the mode-resolved phonon rates used to converge grids,
 * Methods: computational details; Eq. ph-ph differentiated in the destination population):
 *   rates[row(a)] = -dI^{ph-ph}_a/dN_a = sum_em W (N' + N'' + 1) + sum_abs W (N'' - N')
 * over the stored ph-ph channels of each sub-lattice phonon a (W as stored: pair and
 * absorption factors included), at the DEVICE state y (FP64 [n_y]); every other row of the
 * DEVICE output rates (FP64 [n_y]) is 0.  Populations in the compute precision, sums in FP64.
 * At Bose-Einstein populations this is the inverse relaxation time of each phonon.  Enqueued
 * on the context's stream.  Errors: INVALID_ARG, STATE (no channels), CUDA. */
int rtbte_phph_rates(rtbte_ctx *ctx, const double *y, double *rates);

/* Advance the state y (FP64 [n_y_total], caller-owned) from opt->t0 to t_out with the method
 * of `opt`.  y is a device pointer, or a host pointer (pinned memory copies fastest), which
 * the call stages through a context buffer: copied to the device first and the result copied
 * back before it returns.  All stepping, error norms and step-size control run on the device:
 * each integration span is one launch of a CUDA graph whose WHILE node repeats the attempt
 * kernels until every instance is done (at most opt->chunk attempts per launch), and the host
 * reads the status block once per launch (MRI_ADAPT: the host also reads the slow error
 * norms once per slow attempt and decides it).  On success y holds the
 * solution at t_out; on failure y holds the last accepted state and st->t its time.
 * Synchronises the stream.  Errors: INVALID_ARG, STATE, TOO_MANY_STEPS, STEP_UNDERFLOW,
 * ERR_TEST_FAIL, NONFINITE, CUDA. */
int rtbte_advance_to(rtbte_ctx *ctx, double t_out, double *y, const rtbte_integ *opt, rtbte_stats *st);

/* Sizes of instance `inst` (channel counts are 0 before rtbte_upload_channels). */
int rtbte_get_sizes(const rtbte_ctx *ctx, int inst, rtbte_sizes *out);

/* Logical channel entries per state row of instance `inst` (host int64 [n_c + n_ph]: an
 * electron row counts its e-ph entries, a phonon row its ph-e and ph-ph entries), after
 * rtbte_upload_channels in any mode (RTBTE_CH_COUNT included); rows outside a context's row
 * slice count 0 unless the mode was RTBTE_CH_COUNT.  The cost weights for balancing row
 * slices.  Errors: INVALID_ARG, STATE (nothing counted yet). */
int rtbte_row_entries(const rtbte_ctx *ctx, int inst, int64_t *counts);

/* Copy instance `inst`'s stored lists back to host in the PREBUILT logical order (padding
 * removed; q-blocked e-ph lists are merged back into segments (mode, electron, process) with
 * sources ascending).  which: RTBTE_EPH, RTBTE_PHE or RTBTE_PHPH.  off must hold the segment
 * count + 1 entries (e-ph 2*nmodes*n_c, ph-e n_ph, ph-ph 2*n_pp); a/b/W must hold the logical
 * entry count (rtbte_get_sizes).  For e-ph a/b are (src, phonon); ph-e (dst, src); ph-ph
 * (b, c).  Synchronous. */
/* The same for the segments [seg_begin, seg_end) of that order only (for lists too large to
 * copy back whole): off receives seg_end - seg_begin + 1 offsets relative to the first; with
 * a = NULL only off is filled (to size a/b/W), else a/b/W hold `cap` entries at most.
 * Synchronous.  Errors: INVALID_ARG (range, capacity), STATE (no channels), CUDA. */
int rtbte_download_segments(rtbte_ctx *ctx, int inst, unsigned which, int64_t seg_begin, int64_t seg_end, int64_t *off,
                            int32_t *a, int32_t *b, double *W, int64_t cap);
int rtbte_download_channels(rtbte_ctx *ctx, int inst, unsigned which, int64_t *off, int32_t *a, int32_t *b,
                            double *W);

/* Set the stream used by later calls (cudaStream_t; NULL = default stream). */
int rtbte_set_stream(rtbte_ctx *ctx, void *stream);

/* Autotuner of the collision kernel's launch.  The persistent launch divides the work items
 * among CTAs by weight = (entries + w) x c_part per item, w being the fixed cost of an item in
 * entry equivalents and c_part the calibrated cost of an entry of each part; a share s of the
 * weight is split statically, the rest is taken in chunks by CTAs that finish early; each
 * warp prefetches the entry arrays of the item d positions ahead of its sequence into L2.
 * In FP32 the kernel also has two launch forms, two register buffers of entries per warp at 16
 * warps per SM or one buffer at 24 warps per SM, chosen per parts mask.
 * This call times the kernel for `parts` over the forms and candidates of w, c_part, d and s and
 * keeps the fastest for that parts mask (w in *chosen when not NULL); masks never tuned
 * themselves take its w, c_part, d and s.  Each parts mask keeps its own parameters, so tuning
 * the fast and slow masks of MRI does not change the full-RHS launch.  Synchronises the stream;
 * results of later calls do not depend on the choice (rows add item partials in a fixed order).
 * Errors: INVALID_ARG, STATE, CUDA. */
int rtbte_autotune(rtbte_ctx *ctx, unsigned parts, int *chosen);

/* The launch parameters of the full-RHS mask (RTBTE_ALL): w, d and s as described for
 * rtbte_autotune (any pointer may be NULL).  Errors: INVALID_ARG. */
int rtbte_get_tuning(const rtbte_ctx *ctx, int32_t *item_weight, int32_t *prefetch_items, double *static_share);

/* How rtbte_advance_to runs attempts: 1 (default) as one launch of the device-loop CUDA graph
 * per span; 0 as direct kernel launches, one attempt per host check (same kernels and results,
 * slower; for per-kernel profiling tools that do not descend into graph loops).
 * Errors: INVALID_ARG. */
int rtbte_set_graph_mode(rtbte_ctx *ctx, int use_graphs);

/* Kernel timing.  While enabled, every launch of the collision kernel enqueued outside a
 * CUDA graph (rtbte_rhs and the first-step estimate) is bracketed by CUDA events recorded on
 * the context stream.  rtbte_kernel_time synchronises the stream and returns the summed
 * device time (ms) and the number of timed launches since the previous query (then resets).
 * rtbte_advance_to replays graphs and is not timed.  Errors: INVALID_ARG, CUDA. */
int rtbte_set_kernel_timing(rtbte_ctx *ctx, int enable);
int rtbte_kernel_time(rtbte_ctx *ctx, double *total_ms, int64_t *launches);

/* Number of kernel launches the library enqueued since the context was created. */
int64_t rtbte_launch_count(const rtbte_ctx *ctx);

/* Message of the last failure on this context (never NULL). */
const char *rtbte_last_error(const rtbte_ctx *ctx);
const char *rtbte_status_string(int status);

/* ---- allocation-free e-ph RHS ----------------------------------------------------------
 * The paper has no counterpart to this entry point.  It exists for callers that cannot
 * allocate device memory: programs whose device memory is owned entirely by another
 * allocator or by an arena reserved at start-up (a serving runtime, a host application that
 * budgets every byte of the GPU), and latency-critical loops where an allocation's implicit
 * synchronisation is not acceptable.  It needs no context and calls no cudaMalloc, cudaFree
 * or other allocating routine.
 *
 * Writes ydot[0..n_c) = I^{e-ph} (the electron rows of one instance) from caller-owned
 * device arrays: y (FP64 [n_c + n_ph], the instance's state vector) and the e-ph channel
 * list in the layout rtbte_download_channels(RTBTE_EPH) returns -- off (int64
 * [2*nmodes*n_c + 1], segment (nu*n_c + d)*2 + proc), src (int32 source electron), ph (int32
 * full phonon index, < n_ph), W (FP64 weights) -- into ydot (FP64 [n_c]).  Arithmetic as in
 * RTBTE_PREC_FP32_COMP.  Working memory is one fixed array of RTBTE_NOALLOC_SCRATCH_BYTES in
 * the library's device image (held by every device that loads the library until exit);
 * sizes needing more (4 B per state row, each part rounded up to 16 B, plus 8 B per list
 * segment) are rejected with RTBTE_E_UNSUPPORTED before any work.  The first call on a
 * device looks that array up (cudaGetSymbolAddress, which may load the library's device
 * code): make it before any stream capture on that device.  All calls on a device share the
 * array, so calls that can overlap on the GPU (other streams, other host threads) race:
 * serialise them.  Enqueued on `stream` (a cudaStream_t), asynchronous.
 * Errors: INVALID_ARG (bad size or NULL pointer), UNSUPPORTED (too large), CUDA. */
#define RTBTE_NOALLOC_SCRATCH_BYTES (8u << 20)
int rtbte_eph_rhs_noalloc(int32_t n_c, int64_t n_ph, int32_t nmodes, const int64_t *off, const int32_t *src,
                          const int32_t *ph, const double *W, const double *y, double *ydot, void *stream);

/* ---------------------------------------------------------------------------------------
 * Neural-operator surrogate of the ph-ph integral (the learned part of this library; the
 * paper has none).  A periodic-convolution network maps the phonon populations of one
 * instance's ph-ph sub-lattice (one channel per branch, nq_s[0] x nq_s[1], 2-D models only)
 * to I^{ph-ph} (Eq. ph-ph) on that sub-lattice:
 *   x = (N - mu)/sd;  h_l = tanh(conv3x3_periodic(h_{l-1}) + b_l), l = 1..4 (C -> w -> w -> w -> w);
 *   h5 = tanh(h4 M1 + c1);  out = h5 M2 + c2;  I = out * so      (C = nmodes, w = width)
 * Training and inference run on the GPU: every product is a BF16 tensor-core GEMM with FP32
 * accumulation; master weights, Adam moments and activations are FP32.  Parameters in the
 * logical order W1 [9, C, w], b1 [w], W2 [9, w, w], b2, W3, b3, W4, b4, M1 [w, w], c1 [w],
 * M2 [w, C], c2 [C] (row-major; tap = (dy+1)*3 + (dx+1), tap input (y+dy, x+dx) mod n).
 * Sample arrays are [B, nq_s[1], nq_s[0], C] (x fastest, channel innermost). */
typedef struct rtbte_surrogate rtbte_surrogate;

/* Create a surrogate for instance `inst` of `ctx` (which must outlive it): width w (multiple
 * of 8, 8..256), room for `capacity` collected pairs, weights N(0, 1/fan_in) from `seed`
 * (last layer x0.1), biases 0.  Errors: INVALID_ARG, UNSUPPORTED (no sub-lattice, dim != 2,
 * more than 16 branches), OOM/CUDA. */
int rtbte_surrogate_create(rtbte_ctx *ctx, int inst, int width, int capacity, uint64_t seed, rtbte_surrogate **out);

/* Evaluate the exact slow part (RTBTE_SLOW) at the DEVICE state y (FP64 [n_y]) and store the
 * pair (N, I^{ph-ph}) of the surrogate's instance, in FP32, on the device, tagged with the
 * caller's trajectory id (pairs are numbered in collection order).  Enqueued on the context's
 * stream.  Errors: INVALID_ARG (NULL or buffer full), those of rtbte_rhs. */
int rtbte_surrogate_collect(rtbte_surrogate *s, const double *y, int trajectory);

/* `steps` Adam steps (beta 0.9/0.999, eps 1e-8, learning rate lr), each on `batch` training
 * units drawn without replacement per epoch (seeded shuffle).  horizon = 0: a unit is one
 * collected pair and the loss is mean((out - I/so)^2).  horizon > 0: a unit is two pairs i < j
 * of one trajectory with j - i <= horizon and the loss is the mean square of
 * (out_j - out_i) - (I_j - I_i)/so, the quantity the control variate uses.  The first call fixes
 * the per-channel normalisation (mu, sd of N; so = RMS of I) from the pairs collected so far.
 * Synchronises; *loss_out (may be NULL) = the loss of the last minibatch.
 * Errors: INVALID_ARG, STATE (no pairs / no units), OOM/CUDA. */
int rtbte_surrogate_train(rtbte_surrogate *s, int steps, int batch, int horizon, float lr, float *loss_out);

/* out (DEVICE FP64 [n_y]) = the surrogate's I^{ph-ph} on the instance's sub-lattice rows and 0
 * on every other row, for the DEVICE state y.  Enqueued on the context's stream. */
int rtbte_surrogate_predict(rtbte_surrogate *s, const double *y, double *out);

/* Loss and gradients for HOST inputs: x, t FP32 [B, nq_s[1], nq_s[0], C], already normalised
 * (x rounded to BF16 on the device).  *loss = mean((out - t)^2); grad (may be NULL) receives
 * rtbte_surrogate_num_params() FP32 values in the logical order; out (may be NULL) receives
 * the network output FP32 [B, ..., C].  Synchronises. */
int rtbte_surrogate_loss_grad(rtbte_surrogate *s, const float *x, const float *t, int B, float *loss, float *grad,
                              float *out);
int64_t rtbte_surrogate_num_params(const rtbte_surrogate *s);
/* Copy the FP32 master weights to / from host memory (logical order); set refreshes the BF16 copy. */
int rtbte_surrogate_get_params(rtbte_surrogate *s, float *host);
int rtbte_surrogate_set_params(rtbte_surrogate *s, const float *host);
/* Normalisation (arrays of nmodes, may be NULL) and the number of collected pairs. */
void rtbte_surrogate_stats(const rtbte_surrogate *s, float *mu, float *sd, float *so, int *count);

/* Use `s` (NULL detaches) for the slow part of RTBTE_METHOD_MRI_KW3 integrations of this
 * context (single-instance contexts; the surrogate's instance must be 0).  Each slow step
 * takes f^s(Y) = I_exact(Y_ref) + S(Y) - S(Y_ref) (control variate about the reference
 * state Y_ref of the last exact evaluation, S = the surrogate).  Every `judge_period` slow
 * steps the exact integral is evaluated at the step's start state: it becomes the new
 * reference, and if the relative 2-norm error of the control-variate value against it
 * exceeds `judge_tol`, the surrogate is detached for the rest of the call (exact slow part;
 * reported in rtbte_stats.surrogate_fallbacks).  Width 64 runs the fused single-sample
 * inference kernels (four launches per value); other widths the training kernels.
 * Errors: INVALID_ARG, STATE (untrained), UNSUPPORTED. */
int rtbte_set_surrogate(rtbte_ctx *ctx, rtbte_surrogate *s, int judge_period, double judge_tol);

/* GEMM engine of the surrogate's training and batched forward passes: 0 (the default where the
 * device has them) = fifth-generation tensor cores (tcgen05.mma, accumulator in tensor memory,
 * operand tiles by TMA with 128-byte swizzle) for the forward layers, the input gradients and
 * (widths that are multiples of 64) the weight gradients; mma.sync for the rest; 1 = mma.sync for
 * every product.  Both use BF16 operands and FP32 accumulation.  Errors: INVALID_ARG,
 * UNSUPPORTED (engine 0 on a device without tcgen05), STATE. */
int rtbte_surrogate_set_gemm(rtbte_surrogate *s, int engine);

/* Release the surrogate's device memory (NULL is ignored). */
void rtbte_surrogate_destroy(rtbte_surrogate *s);

/* Release every device and host resource of the context (NULL is ignored). */
void rtbte_destroy(rtbte_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* RTBTE_H */
