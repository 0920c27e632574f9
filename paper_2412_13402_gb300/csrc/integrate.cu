// integrate.cu -- time integration of the rt-BTE on the device (Methods B).
//
// One attempted step of an explicit RK method (Eq. ERK_method) is a fixed kernel sequence:
//   prep      populations <- y                                  (stage 1: z_1 = y)
//   S times:  collision kernel (rhs.cu) -> partials per work item
//             stage kernel: k_i = -sum(partials) [+ MRI forcing];  z_{i+1} = y + h sum_j A_{i+1,j} k_j
//             written straight into the population copies; after the last stage
//             y_new = y + h sum b_i k_i, e = h sum (b_i - bt_i) k_i and per-block WRMS partials
//             of e with weights 1/(rtol |y_{n-1}| + atol_i) (Eqs. wrms_norm, wrms_weights)
//   controller (one block): WRMS norm in a fixed order, accept if <= 1, PID step proposal
//             h' = h eps_k^{-a1/p} eps_{k-1}^{+a2/p} eps_{k-2}^{-a3/p} (Eq. pid_controller)
// Step size, time, error history and which of two state buffers is current live in device
// memory, so the sequence is captured once into a CUDA graph whose WHILE conditional node
// repeats it on the device until every instance is done (at most a cap of attempts per
// launch); the host reads a small status block once per launch.  Readings of what the paper leaves
// open: PID signs alternate (ARKODE's documented form; the printed all-negative form is
// pid_sign_mode 1), the other controller constants are ARKODE's documented defaults, the
// first step follows Hairer-Norsett-Wanner's starting-step algorithm, and the MIS coupling
// of the last MRI stage is b_j - A_{S,j} (the printed A_{S-1,j} does not reduce MIS to its
// base method when the fast part vanishes).
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"
#include "rows.cuh"

namespace rtbte {

RowParams row_params(rtbte_ctx *ctx);

namespace {

constexpr int kRedThreads = 256;

// ---- Butcher tableaux (as exact fractions in double) --------------------------------
Tableau tableau_of(int method) {
    Tableau T;
    std::memset(&T, 0, sizeof(T));
    if (method == RTBTE_RK4 || method == RTBTE_SPLIT_RK4) {  // classical RK4
        T.S = 4; T.p = 4; T.has_emb = 0;
        T.c[1] = 1.0 / 2; T.c[2] = 1.0 / 2; T.c[3] = 1.0;
        T.A[1][0] = 1.0 / 2; T.A[2][1] = 1.0 / 2; T.A[3][2] = 1.0;
        T.b[0] = 1.0 / 6; T.b[1] = 1.0 / 3; T.b[2] = 1.0 / 3; T.b[3] = 1.0 / 6;
    } else if (method == RTBTE_BS32) {  // Bogacki-Shampine 3(2)
        T.S = 4; T.p = 3; T.has_emb = 1;
        T.c[1] = 1.0 / 2; T.c[2] = 3.0 / 4; T.c[3] = 1.0;
        T.A[1][0] = 1.0 / 2;
        T.A[2][1] = 3.0 / 4;
        T.A[3][0] = 2.0 / 9; T.A[3][1] = 1.0 / 3; T.A[3][2] = 4.0 / 9;
        T.b[0] = 2.0 / 9; T.b[1] = 1.0 / 3; T.b[2] = 4.0 / 9; T.b[3] = 0.0;
        T.bt[0] = 7.0 / 24; T.bt[1] = 1.0 / 4; T.bt[2] = 1.0 / 3; T.bt[3] = 1.0 / 8;
    } else {  // Zonneveld 4(3)
        T.S = 5; T.p = 4; T.has_emb = 1;
        T.c[1] = 1.0 / 2; T.c[2] = 1.0 / 2; T.c[3] = 1.0; T.c[4] = 3.0 / 4;
        T.A[1][0] = 1.0 / 2;
        T.A[2][1] = 1.0 / 2;
        T.A[3][2] = 1.0;
        T.A[4][0] = 5.0 / 32; T.A[4][1] = 7.0 / 32; T.A[4][2] = 13.0 / 32; T.A[4][3] = -1.0 / 32;
        T.b[0] = 1.0 / 6; T.b[1] = 1.0 / 3; T.b[2] = 1.0 / 3; T.b[3] = 1.0 / 6; T.b[4] = 0.0;
        T.bt[0] = -1.0 / 2; T.bt[1] = 7.0 / 3; T.bt[2] = 7.0 / 3; T.bt[3] = 13.0 / 6; T.bt[4] = -16.0 / 3;
    }
    return T;
}

// Knoth-Wolke 3-stage base of the MIS method and its MRI abscissae / couplings (K = 1).
struct Mis {
    double chat[4];
    double Om[4][3];
};
Mis mis_kw3() {
    const double A[3][3] = {{0, 0, 0}, {1.0 / 3, 0, 0}, {-3.0 / 16, 15.0 / 16, 0}};
    const double b[3] = {1.0 / 6, 3.0 / 10, 8.0 / 15};
    const double c[3] = {0, 1.0 / 3, 3.0 / 4};
    Mis M;
    std::memset(&M, 0, sizeof(M));
    for (int i = 0; i < 3; ++i) M.chat[i] = c[i];
    M.chat[3] = 1.0;
    for (int i = 1; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M.Om[i][j] = A[i][j] - A[i - 1][j];
    for (int j = 0; j < 3; ++j) M.Om[3][j] = b[j] - A[2][j];
    return M;
}

struct StageArgs {
    Tableau T;
    CtlParams cp;
    Ctl *ctl;  // one controller per instance
    double *Y0, *Y1, *K;
    const double *forcing;
    double *wsq;  // per-row squared weighted error of the last stage
    unsigned long long *range;  // per instance: rows of the attempted state out of range
    long long n;
    unsigned parts;
    int stage;         // -1: populations <- y; 0..S-1: combine stage `stage`
    int respect_done;  // inside an attempt sequence: skip instances whose integration is done
    int batched;       // several instances: rows visited by row blocks of active instances only
};

__device__ __forceinline__ double atol_of(const CtlParams &cp, const InstDev &I, long long local) {
    return local < I.n_c ? cp.atol_c : cp.atol_ph;
}

template <class R>
__device__ __forceinline__ void stage_row(const RowParams &Q, const StageArgs &a, int ii, const InstDev &I, long long c) {
    const int S = a.T.S, i = a.stage;
    const Ctl *C = a.ctl + ii;
    const long long local = c - I.y_off;
    const double *y = C->cur ? a.Y1 : a.Y0;
    if (i < 0) {
        write_pops<R>(Q, I, local, y[c]);
        return;
    }
    const double h = C->h_try;
    double k = row_value<R>(Q, I, local, a.parts);
    if (a.forcing) k += a.forcing[c];
    a.K[(long long)i * a.n + c] = k;
    if (i < S - 1) {
        double acc = 0.0;
        for (int j = 0; j <= i; ++j) acc += a.T.A[i + 1][j] * a.K[(long long)j * a.n + c];
        write_pops<R>(Q, I, local, (R)(y[c] + h * acc));
    } else {
        double s1 = 0.0, s2 = 0.0;
        for (int j = 0; j < S; ++j) {
            const double kj = a.K[(long long)j * a.n + c];
            s1 += a.T.b[j] * kj;
            s2 += (a.T.b[j] - a.T.bt[j]) * kj;
        }
        const double ynew = y[c] + h * s1;
        (C->cur ? a.Y0 : a.Y1)[c] = ynew;
        // populations outside their physical range (f in [0,1], N >= 0) beyond the absolute
        // tolerance: counted per attempt, added to the instance's total if it is accepted
        const bool out = local < I.n_c ? (ynew < -a.cp.atol_c || ynew > 1.0 + a.cp.atol_c) : (ynew < -a.cp.atol_ph);
        if (out && a.range) atomicAdd(a.range + ii, 1ULL);
        double x2 = 0.0;
        if (a.T.has_emb) {  // error weight and weighted error in FP64 (step acceptance reads them)
            const double w = 1.0 / (a.cp.rtol * fabs(y[c]) + atol_of(a.cp, I, local));
            const double x = h * s2 * w;
            x2 = x * x;
        }
        if (!isfinite(ynew)) x2 = __longlong_as_double(0x7ff8000000000000LL);
        a.wsq[c] = x2;
    }
}

// Exclusive prefix of v over the threads of the block (thread order); *total = the block's sum.
// Called by every thread of the block, once per kernel.
__device__ int block_excl_scan(int v, int *total) {
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nw ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) ws[lane] = w;
    }
    __syncthreads();
    *total = ws[nw - 1];
    return incl - v + (wid > 0 ? ws[wid - 1] : 0);
}

// Stage combination over the rows.  Several instances: every block first lists the row blocks
// (kRedThreads rows of one instance, one row per thread) of the instances still integrating --
// a prefix over instances in shared memory -- and the grid walks only those, so a launch late in
// a batched integration, with a few slow instances left, costs their rows and nothing else.  One
// instance: a grid-stride loop over its rows.
template <class R>
__global__ void __launch_bounds__(kRedThreads) stage_kernel(RowParams Q, StageArgs a) {
    if (a.batched) {
        __shared__ int s_pre[kMaxBatch + 1];  // s_pre[i]: first active row block of instance i
        const int NI = Q.n_inst;              // <= kMaxBatch (checked on the host)
        const int C = (NI + blockDim.x - 1) / blockDim.x;
        const int i0 = threadIdx.x * C;
        int run = 0;
        for (int i = i0; i < i0 + C && i < NI; ++i) {
            if (!(a.respect_done && a.ctl[i].done)) {
                const long long rows = (long long)Q.inst[i].n_c + Q.inst[i].n_ph;
                run += (int)((rows + kRedThreads - 1) / kRedThreads);
            }
            s_pre[i + 1] = run;
        }
        int total;
        const int before = block_excl_scan(run, &total);
        for (int i = i0; i < i0 + C && i < NI; ++i) s_pre[i + 1] += before;
        if (threadIdx.x == 0) s_pre[0] = 0;
        __syncthreads();
        for (int b = blockIdx.x; b < total; b += gridDim.x) {
            int lo = 0, hi = NI - 1;  // the last instance with s_pre[i] <= b (an active one)
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_pre[mid] <= b) lo = mid; else hi = mid - 1;
            }
            const InstDev I = Q.inst[lo];
            const long long r = (long long)(b - s_pre[lo]) * kRedThreads + threadIdx.x;
            if (r < (long long)I.n_c + I.n_ph) stage_row<R>(Q, a, lo, I, I.y_off + r);
        }
        return;
    }
    const InstDev I = Q.inst[0];
    if (a.respect_done && a.ctl[0].done) return;
    // 32-row chunks dealt round-robin over the blocks (warp w of block b takes chunk w * grid + b
    // first), so that the electron rows, which sum many more item partials than phonon rows and
    // come first in the state, spread over every SM instead of filling the first blocks
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long nch = (a.n + 31) >> 5;
    for (long long ch = (long long)w * gridDim.x + blockIdx.x; ch < nch; ch += (long long)gridDim.x * nw) {
        const long long c = (ch << 5) + lane;
        if (c < a.n) stage_row<R>(Q, a, 0, I, c);
    }
}

// Fixed-order sum of v[b .. b+n) by one block: strided per-thread sums, a butterfly within each
// warp (both partners of a pair add the same two values, so every lane holds the same bits), then
// the warp sums in warp order.  Every thread returns the sum.
__device__ double block_sum(const double *v, long long b, long long n) {
    __shared__ double ws[kRedThreads / 32];
    double acc = 0.0;
    for (long long r = threadIdx.x; r < n; r += blockDim.x) acc += v[b + r];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += ws[w];
    __syncthreads();  // ws is free for the next call
    return r;
}

__device__ __forceinline__ void arm(Ctl *c) {
    double hk = c->h;
    c->last = 0;
    if (c->fixed) {  // classical fixed steps: last step ends exactly at t_out
        c->last = (c->steps + 1 >= c->max_steps) ? 1 : 0;
        c->h_try = c->last ? c->t_out - c->t : hk;
        return;
    }
    if (c->t + hk >= c->t_out) {
        hk = c->t_out - c->t;
        c->last = 1;
    }
    c->h_try = hk;
}

// One block per instance: WRMS norm (Eq. wrms_norm) of its rows, accept/reject, PID proposal.
// Per-instance partial sums of a state-size vector: block (c, i) adds chunk c of instance i's
// rows (fixed chunk boundaries and order, so the norms are deterministic); finished instances
// are skipped when respect_done.
__global__ void wrms_chunks(RowParams Q, const Ctl *ctl, const double *wsq, double *part, int respect_done) {
    const int i = blockIdx.y;
    if (respect_done && ctl[i].done) return;
    const InstDev I = Q.inst[i];
    const long long ni = (long long)I.n_c + I.n_ph;
    const long long L = (ni + gridDim.x - 1) / gridDim.x;
    const long long b = (long long)blockIdx.x * L;
    const long long e = b + L < ni ? b + L : ni;
    const double s = block_sum(wsq, I.y_off + b, e > b ? e - b : 0);
    if (threadIdx.x == 0) part[(long long)i * gridDim.x + blockIdx.x] = s;
}

__global__ void controller_kernel(RowParams Q, Ctl *ctl, CtlParams cp, const double *part,
                                  unsigned long long *range) {
    Ctl *c = ctl + blockIdx.x;
    if (c->done) return;
    const InstDev I = Q.inst[blockIdx.x];
    const long long ni = (long long)I.n_c + I.n_ph;
    const double sum = block_sum(part, (long long)blockIdx.x * kWrmsChunks, kWrmsChunks);
    if (threadIdx.x >= 32) return;
    const double eps = sqrt(sum / (double)ni);
    // logarithms of the three PID factors, one per lane, ahead of the scalar logic of thread 0:
    // FP64 transcendental functions are slow in a single thread on this GPU, and the three are
    // independent (lane 0: the floored error norm, lanes 1-2: the two previous ones)
    double lg = 0.0;
    if (threadIdx.x < 3) lg = log(threadIdx.x == 0 ? fmax(eps, 1e-10) : threadIdx.x == 1 ? c->eps1 : c->eps2);
    const double lg1 = __shfl_sync(0xffffffffu, lg, 1), lg2 = __shfl_sync(0xffffffffu, lg, 2);
    if (threadIdx.x != 0) return;
    const double lg0 = lg;
    const unsigned long long nr = range[blockIdx.x];
    range[blockIdx.x] = 0;
    c->attempts++;
    if (!isfinite(eps)) {
        c->status = RTBTE_E_NONFINITE;
        c->done = 1;
        return;
    }
    if (c->fixed) {
        c->cur ^= 1;
        c->t = c->last ? c->t_out : c->t + c->h_try;
        c->steps++;
        c->range_viol += (long long)nr;
        c->h_last = c->h_try;
        if (c->last) c->done = 1;
        else arm(c);
        return;
    }
    const double p = (double)cp.p;
    c->eps = eps;
    if (eps <= 1.0) {
        c->cur ^= 1;
        c->t = c->last ? c->t_out : c->t + c->h_try;
        c->steps++;
        c->range_viol += (long long)nr;
        const double e = eps > 1e-10 ? eps : 1e-10;
        // e^(-a1/p) eps1^(+-a2/p) eps2^(-a3/p) as one exponential of the lanes' logarithms
        const double x2 = cp.pid_sign_mode == 0 ? cp.a2 / p : -cp.a2 / p;
        double eta = exp((-cp.a1 / p) * lg0 + x2 * lg1 + (-cp.a3 / p) * lg2);
        eta *= cp.safety;
        double cap = c->first ? cp.growth_first : cp.growth;
        if (c->nef > 0 && cap > 1.0) cap = 1.0;
        if (eta > cap) eta = cap;
        double h = c->h_try * eta;
        if (cp.hmax > 0 && h > cp.hmax) h = cp.hmax;
        c->h = h;
        c->eps2 = c->eps1;
        c->eps1 = e;
        c->first = 0;
        c->nef = 0;
        c->h_last = c->h_try;
        if (c->t >= c->t_out) {
            c->done = 1;
            return;
        }
        if (!(c->t + h > c->t)) {  // the proposed step no longer advances time
            c->status = RTBTE_E_STEP_UNDERFLOW;
            c->done = 1;
            return;
        }
        if (c->steps - c->steps_base >= c->max_steps) {
            c->status = RTBTE_E_TOO_MANY_STEPS;
            c->done = 1;
            return;
        }
    } else {
        c->fails++;
        c->nef++;
        if (c->nef >= cp.max_nef) {
            c->status = RTBTE_E_ERR_TEST_FAIL;
            c->done = 1;
            return;
        }
        double eta = cp.safety * exp((-1.0 / p) * lg0);  // eps^(-1/p); eps > 1 here, so lg0 = log(eps)
        if (eta < cp.etamin) eta = cp.etamin;
        if (eta > 1.0) eta = 1.0;
        if (c->nef >= cp.small_nef && eta > cp.etamxf) eta = cp.etamxf;
        const double h = c->h_try * eta;
        c->h = h;
        if (h < cp.hmin || !(c->t + h > c->t)) {
            c->status = RTBTE_E_STEP_UNDERFLOW;
            c->done = 1;
            return;
        }
    }
    arm(c);
}

// ---- Hairer-Norsett-Wanner starting step, per instance --------------------------------
__global__ void __launch_bounds__(kRedThreads) h0_norms(RowParams Q, CtlParams cp, const Ctl *ctl, const double *Y0,
                                                         const double *Y1, const double *K0, const double *K1,
                                                         double *wsq, int second, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int ii = Q.n_inst > 1 ? find_inst(Q, c) : 0;
        const InstDev I = Q.inst[ii];
        const double *y = ctl[ii].cur ? Y1 : Y0;
        const double w = 1.0 / (cp.rtol * fabs(y[c]) + atol_of(cp, I, c - I.y_off));
        if (!second) {
            const double a = y[c] * w, b = K0[c] * w;
            wsq[c] = a * a;
            wsq[n + c] = b * b;
        } else {
            const double d = (K1[c] - K0[c]) * w;
            wsq[c] = d * d;
        }
    }
}

__global__ void h0_first(RowParams Q, Ctl *ctl, const double *part0, const double *part1, double span) {
    Ctl *c = ctl + blockIdx.x;
    const InstDev I = Q.inst[blockIdx.x];
    const long long ni = (long long)I.n_c + I.n_ph;
    const double s0 = block_sum(part0, (long long)blockIdx.x * kWrmsChunks, kWrmsChunks);
    const double s1 = block_sum(part1, (long long)blockIdx.x * kWrmsChunks, kWrmsChunks);
    if (threadIdx.x != 0) return;
    const double d0 = sqrt(s0 / (double)ni), d1 = sqrt(s1 / (double)ni);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    if (h0 > span) h0 = span;
    c->h0tmp = h0;
    c->eps = d1;  // kept for the second half
}

template <class R>
__global__ void h0_probe(RowParams Q, const Ctl *ctl, const double *Y0, const double *Y1, const double *K0, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int ii = Q.n_inst > 1 ? find_inst(Q, c) : 0;
        const InstDev I = Q.inst[ii];
        const double *y = ctl[ii].cur ? Y1 : Y0;
        write_pops<R>(Q, I, c - I.y_off, y[c] + ctl[ii].h0tmp * K0[c]);
    }
}

__global__ void h0_second(RowParams Q, Ctl *ctl, CtlParams cp, const double *part, double span) {
    Ctl *c = ctl + blockIdx.x;
    const InstDev I = Q.inst[blockIdx.x];
    const long long ni = (long long)I.n_c + I.n_ph;
    const double s = block_sum(part, (long long)blockIdx.x * kWrmsChunks, kWrmsChunks);
    if (threadIdx.x != 0) return;
    const double h0 = c->h0tmp, d1 = c->eps;
    const double d2 = sqrt(s / (double)ni) / h0;
    const double dm = d1 > d2 ? d1 : d2;
    const double h1 = dm <= 1e-15 ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 1.0 / (cp.p + 1));
    double h = 100.0 * h0 < h1 ? 100.0 * h0 : h1;
    if (h > span) h = span;
    if (cp.hmax > 0 && h > cp.hmax) h = cp.hmax;
    c->h = h;
    c->eps = 0.0;
    arm(c);
}

__global__ void arm_kernel(Ctl *ctl, int n_inst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_inst) arm(ctl + i);
}

// Inner (fast) ERK restart for an MRI stage: fresh error history, carried step proposal.
__global__ void mri_stage_reset(Ctl *ctl, int n_inst, CtlParams cp, double ta, double tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    Ctl *c = ctl + i;
    c->t = ta;
    c->t_out = tb;
    c->eps1 = 1.0;
    c->eps2 = 1.0;
    c->first = 1;
    c->nef = 0;
    c->done = 0;
    c->status = 0;
    c->steps_base = c->steps;
    double h = c->h;
    if (h > tb - ta) h = tb - ta;
    if (cp.hmax > 0 && h > cp.hmax) h = cp.hmax;
    c->h = h;
    if (h > 0) arm(c);
}

// MIS forcing of stage i (Methods B, step 2b with K = 1): r = (1/dc_i) sum_{j<i} Om_ij fs_j
__global__ void mri_forcing(double *r, const double *Fs, double om0, double om1, double om2, int i, double dc,
                            long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        const double om[3] = {om0, om1, om2};
        for (int j = 0; j < i; ++j) acc += om[j] * Fs[(long long)j * n + c];
        r[c] = acc / dc;
    }
}

// Tolerance-chosen MRI (step doubling on the MIS step): copy each instance's rows between its
// current state buffer and buf (to_buf: current -> buf, else buf -> current).
__global__ void copy_cur(RowParams Q, const Ctl *ctl, double *Y0, double *Y1, double *buf, long long n, int to_buf) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int ii = Q.n_inst > 1 ? find_inst(Q, c) : 0;
        double *y = ctl[ii].cur ? Y1 : Y0;
        if (to_buf) buf[c] = y[c]; else y[c] = buf[c];
    }
}

// Squared weighted local-error estimate of the two-half-step result y_2 (the current state):
// e = (y_1 - y_2) / (2^3 - 1) for the order-3 slow method, weights from y_n (Eq. wrms_weights).
__global__ void __launch_bounds__(kRedThreads) slow_err_sq(RowParams Q, CtlParams cp, const Ctl *ctl, const double *Y0,
                                                             const double *Y1, const double *yn, const double *y1,
                                                             double *wsq, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int ii = Q.n_inst > 1 ? find_inst(Q, c) : 0;
        const InstDev I = Q.inst[ii];
        const double y2 = (ctl[ii].cur ? Y1 : Y0)[c];
        const double w = 1.0 / (cp.rtol * fabs(yn[c]) + atol_of(cp, I, c - I.y_off));
        const double d = (y1[c] - y2) / 7.0 * w;
        wsq[c] = d * d;
    }
}

// Per-instance WRMS norm (Eq. wrms_norm) from the chunk sums of wrms_chunks.
__global__ void slow_eps(RowParams Q, const double *part, double *eps) {
    const InstDev I = Q.inst[blockIdx.x];
    const long long ni = (long long)I.n_c + I.n_ph;
    const double sum = block_sum(part, (long long)blockIdx.x * kWrmsChunks, kWrmsChunks);
    if (threadIdx.x == 0) eps[blockIdx.x] = sqrt(sum / (double)ni);
}

// ---- host helpers -----------------------------------------------------------------------
int row_grid(rtbte_ctx *ctx) { return (int)std::min<long long>((ctx->n_y + kRedThreads - 1) / kRedThreads, kWrmsBlocks); }
int n_inst(rtbte_ctx *ctx) { return (int)ctx->inst.size(); }

template <class R>
int launch_stage(rtbte_ctx *ctx, const StageArgs &a, cudaStream_t s) {
    const long long want = a.batched ? ctx->n_rblk : (ctx->n_y + kRedThreads - 1) / kRedThreads;
    const int grid = (int)std::max<long long>(1, std::min<long long>(want, ctx->stage_resident > 0 ? ctx->stage_resident
                                                                                               : 2 * ctx->num_sms));
    stage_kernel<R><<<grid, kRedThreads, 0, s>>>(row_params(ctx), a);
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    return RTBTE_OK;
}

int stage(rtbte_ctx *ctx, const StageArgs &a, cudaStream_t s) {
    return ctx->precision == RTBTE_PREC_FP64 ? launch_stage<double>(ctx, a, s) : launch_stage<float>(ctx, a, s);
}

StageArgs stage_args(rtbte_ctx *ctx, const Tableau &T, const CtlParams &cp, unsigned parts, const double *forcing) {
    StageArgs a;
    std::memset(&a, 0, sizeof(a));
    a.T = T;
    a.cp = cp;
    a.ctl = ctx->ctl.as<Ctl>();
    a.Y0 = ctx->Y[0].as<double>();
    a.Y1 = ctx->Y[1].as<double>();
    a.K = ctx->K.as<double>();
    a.range = ctx->range_scratch.as<unsigned long long>();
    a.forcing = forcing;
    a.wsq = ctx->wrms_part.as<double>();
    a.n = ctx->n_y;
    a.parts = parts;
    a.batched = n_inst(ctx) > 1 ? 1 : 0;
    return a;
}

// Enqueue one attempted step (prep, S x [collision kernel, stage kernel], controller).
int enqueue_attempt(rtbte_ctx *ctx, const Tableau &T, const CtlParams &cp, unsigned parts, const double *forcing,
                    cudaStream_t s) {
    StageArgs a = stage_args(ctx, T, cp, parts, forcing);
    a.stage = -1;
    a.respect_done = 1;
    int rc;
    if ((rc = stage(ctx, a, s))) return rc;
    for (int i = 0; i < T.S; ++i) {
        if ((rc = launch_rhs_core(ctx, parts, ctx->ctl.as<Ctl>(), s))) return rc;
        a.stage = i;
        if ((rc = stage(ctx, a, s))) return rc;
    }
    double *chunks = ctx->wrms_part.as<double>() + 2 * ctx->n_y;
    wrms_chunks<<<dim3(kWrmsChunks, n_inst(ctx)), kRedThreads, 0, s>>>(row_params(ctx), ctx->ctl.as<Ctl>(),
                                                                      ctx->wrms_part.as<double>(), chunks, 1);
    controller_kernel<<<n_inst(ctx), kRedThreads, 0, s>>>(row_params(ctx), ctx->ctl.as<Ctl>(), cp, chunks,
                                                          ctx->range_scratch.as<unsigned long long>());
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches += 2;
    return RTBTE_OK;
}

long long graph_key(int method, unsigned parts, bool forcing, const CtlParams &cp, int cap) {
    // the controller constants are captured by value: key them by a hash of their bytes
    unsigned long long h = 1469598103934665603ULL ^ (unsigned long long)cap;
    const unsigned char *b = reinterpret_cast<const unsigned char *>(&cp);
    for (size_t i = 0; i < sizeof(cp); ++i) h = (h ^ b[i]) * 1099511628211ULL;
    return (long long)((h & ~0xffffULL) | ((unsigned long long)method << 8) | (parts << 1) | (forcing ? 1 : 0));
}

// Last node of the attempt loop's body: counts the attempts of this graph launch and keeps the
// loop going while some instance is still integrating and fewer than `cap` attempts have run,
// so the loop ends after at most `cap` attempts whatever the other kernels do.
__global__ void loop_guard(const Ctl *ctl, int n_inst, int *iter, int cap, cudaGraphConditionalHandle h) {
    __shared__ int active;
    if (threadIdx.x == 0) active = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x)
        if (!ctl[i].done) atomicExch(&active, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int it = *iter + 1;
        *iter = it;
        cudaGraphSetConditional(h, (active && it < cap) ? 1u : 0u);
    }
}

// Attempts as one CUDA graph with a device-side loop: a memset zeroes the attempt counter, then
// a WHILE conditional node runs [attempt kernels, loop_guard] until every instance is done or
// `cap` attempts have run.  One launch (and one host check) per call instead of one per batch
// of attempts.  Captured on the private stream, launched on the user stream.
int attempt_graph(rtbte_ctx *ctx, int method, const CtlParams &cp, unsigned parts, const double *forcing, int cap,
                  cudaGraphExec_t *out, int *nlaunch) {
    const Tableau T = tableau_of(method);
    long long key = graph_key(method, parts, forcing != nullptr, cp, cap);
    auto it = ctx->graphs.find(key);
    if (it != ctx->graphs.end()) {
        *out = it->second;
        *nlaunch = ctx->graph_launches[key];
        return RTBTE_OK;
    }
    if (!ctx->loop_iter.p) {
        RT_CUDA(ctx, cudaMalloc(&ctx->loop_iter.p, 16));
        ctx->loop_iter.bytes = 16;
    }
    if (!ctx->loop_iter_host) RT_CUDA(ctx, cudaMallocHost(&ctx->loop_iter_host, sizeof(int)));
    int *iter = ctx->loop_iter.as<int>();
    cudaGraph_t g;
    RT_CUDA(ctx, cudaGraphCreate(&g, 0));
    auto bail = [&](cudaError_t e, const char *what) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e, what);
    };
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return bail(e, "cudaGraphConditionalHandleCreate");
    cudaMemsetParams mp{};
    mp.dst = iter;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 1;
    mp.height = 1;
    mp.pitch = 4;
    cudaGraphNode_t ms, cn;
    if ((e = cudaGraphAddMemsetNode(&ms, g, nullptr, 0, &mp)) != cudaSuccess) return bail(e, "cudaGraphAddMemsetNode");
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    if ((e = cudaGraphAddNode(&cn, g, &ms, nullptr, 1, &np)) != cudaSuccess) return bail(e, "cudaGraphAddNode");
    cudaGraph_t body = np.conditional.phGraph_out[0];
    long long before = ctx->launches;
    e = cudaStreamBeginCaptureToGraph(ctx->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bail(e, "cudaStreamBeginCaptureToGraph");
    int rc = enqueue_attempt(ctx, T, cp, parts, forcing, ctx->cap_stream);
    loop_guard<<<1, 256, 0, ctx->cap_stream>>>(ctx->ctl.as<Ctl>(), n_inst(ctx), iter, cap, h);
    cudaError_t el = cudaGetLastError();
    e = cudaStreamEndCapture(ctx->cap_stream, &body);
    ctx->graph_launches[key] = (int)(ctx->launches - before) + 1;  // kernels per attempt, guard included
    ctx->launches = before;                                       // captured, not executed
    if (rc) {
        cudaGraphDestroy(g);
        return rc;
    }
    if (el != cudaSuccess) return bail(el, "loop_guard launch");
    if (e != cudaSuccess) return bail(e, "cudaStreamEndCapture");
    cudaGraphExec_t ex;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    ctx->graphs[key] = ex;
    *out = ex;
    *nlaunch = ctx->graph_launches[key];
    return RTBTE_OK;
}

int read_ctl(rtbte_ctx *ctx) {
    RT_CUDA(ctx, cudaMemcpyAsync(ctx->ctl_host, ctx->ctl.p, sizeof(Ctl) * n_inst(ctx), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RTBTE_OK;
}

// Stream-ordered copy of the pinned host mirror to the device; the host does not write the
// mirror again before the next read_ctl (which synchronises), so no wait is needed here.
int write_ctl(rtbte_ctx *ctx) {
    RT_CUDA(ctx, cudaMemcpyAsync(ctx->ctl.p, ctx->ctl_host, sizeof(Ctl) * n_inst(ctx), cudaMemcpyHostToDevice,
                                 ctx->stream));
    return RTBTE_OK;
}

bool all_done(rtbte_ctx *ctx) {
    for (int i = 0; i < n_inst(ctx); ++i)
        if (!ctx->ctl_host[i].done) return false;
    return true;
}

long long sum_attempts(rtbte_ctx *ctx) {
    long long a = 0;
    for (int i = 0; i < n_inst(ctx); ++i) a += ctx->ctl_host[i].attempts;
    return a;
}

// Run attempts until every instance is done.  Returns a CUDA/launch error code, else RTBTE_OK
// (the integration status of each instance is in ctx->ctl_host[i].status).  *attempts_out
// receives the instance-attempts performed (one per active instance per attempt).
int run_attempts(rtbte_ctx *ctx, int method, const CtlParams &cp, unsigned parts, const double *forcing, int cap,
                 long long *attempts_out) {
    long long a0 = sum_attempts(ctx);
    int rc;
    if (!ctx->use_graphs) {  // direct launches, one attempt per host check (profilers, debugging)
        const Tableau T = tableau_of(method);
        for (;;) {
            if ((rc = enqueue_attempt(ctx, T, cp, parts, forcing, ctx->stream))) return rc;
            if ((rc = read_ctl(ctx))) return rc;
            if (all_done(ctx)) break;
        }
        if (attempts_out) *attempts_out = sum_attempts(ctx) - a0;
        return RTBTE_OK;
    }
    cudaGraphExec_t ex;
    int nl;
    if ((rc = attempt_graph(ctx, method, cp, parts, forcing, cap, &ex, &nl))) return rc;
    for (;;) {
        RT_CUDA(ctx, cudaGraphLaunch(ex, ctx->stream));
        RT_CUDA(ctx, cudaMemcpyAsync(ctx->loop_iter_host, ctx->loop_iter.p, sizeof(int), cudaMemcpyDeviceToHost,
                                     ctx->stream));
        if ((rc = read_ctl(ctx))) return rc;
        ctx->launches += (long long)*ctx->loop_iter_host * nl;
        if (all_done(ctx)) break;
    }
    if (attempts_out) *attempts_out = sum_attempts(ctx) - a0;
    return RTBTE_OK;
}

// Hairer-Norsett-Wanner first step for every instance; 2 RHS evaluations of `parts` (+ forcing).
int h0_estimate(rtbte_ctx *ctx, const CtlParams &cp, unsigned parts, const double *forcing, double span) {
    const int nb = row_grid(ctx);
    RowParams Q = row_params(ctx);
    Ctl *c = ctx->ctl.as<Ctl>();
    double *K0 = ctx->K.as<double>(), *K1 = K0 + ctx->n_y;
    double *wsq = ctx->wrms_part.as<double>();
    StageArgs a = stage_args(ctx, tableau_of(RTBTE_ZON43), cp, parts, forcing);
    a.stage = -1;
    int rc;
    if ((rc = stage(ctx, a, ctx->stream))) return rc;
    if ((rc = launch_rhs_core(ctx, parts, nullptr, ctx->stream))) return rc;
    if ((rc = launch_rows(ctx, parts, K0, forcing, ctx->stream))) return rc;
    double *part0 = wsq + 2 * ctx->n_y, *part1 = part0 + (long long)kWrmsChunks * n_inst(ctx);
    const dim3 cg(kWrmsChunks, n_inst(ctx));
    h0_norms<<<nb, kRedThreads, 0, ctx->stream>>>(Q, cp, c, ctx->Y[0].as<double>(), ctx->Y[1].as<double>(), K0, K1,
                                                  wsq, 0, ctx->n_y);
    wrms_chunks<<<cg, kRedThreads, 0, ctx->stream>>>(Q, c, wsq, part0, 0);
    wrms_chunks<<<cg, kRedThreads, 0, ctx->stream>>>(Q, c, wsq + ctx->n_y, part1, 0);
    h0_first<<<n_inst(ctx), kRedThreads, 0, ctx->stream>>>(Q, c, part0, part1, span);
    if (ctx->precision == RTBTE_PREC_FP64)
        h0_probe<double><<<nb, kRedThreads, 0, ctx->stream>>>(Q, c, ctx->Y[0].as<double>(), ctx->Y[1].as<double>(), K0,
                                                              ctx->n_y);
    else
        h0_probe<float><<<nb, kRedThreads, 0, ctx->stream>>>(Q, c, ctx->Y[0].as<double>(), ctx->Y[1].as<double>(), K0,
                                                             ctx->n_y);
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches += 5;
    if ((rc = launch_rhs_core(ctx, parts, nullptr, ctx->stream))) return rc;
    if ((rc = launch_rows(ctx, parts, K1, forcing, ctx->stream))) return rc;
    h0_norms<<<nb, kRedThreads, 0, ctx->stream>>>(Q, cp, c, ctx->Y[0].as<double>(), ctx->Y[1].as<double>(), K0, K1,
                                                  wsq, 1, ctx->n_y);
    wrms_chunks<<<cg, kRedThreads, 0, ctx->stream>>>(Q, c, wsq, part0, 0);
    h0_second<<<n_inst(ctx), kRedThreads, 0, ctx->stream>>>(Q, c, cp, part0, span);
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches += 3;
    return RTBTE_OK;
}

CtlParams ctl_params(const rtbte_integ *o, int p) {
    CtlParams cp;
    std::memset(&cp, 0, sizeof(cp));
    cp.rtol = o->rtol;
    cp.atol_c = o->atol_c;
    cp.atol_ph = o->atol_ph;
    cp.a1 = o->a1;
    cp.a2 = o->a2;
    cp.a3 = o->a3;
    cp.safety = o->safety > 0 ? o->safety : 0.96;
    cp.growth = o->growth > 0 ? o->growth : 20.0;
    cp.growth_first = o->growth_first > 0 ? o->growth_first : 1e4;
    cp.etamxf = o->etamxf > 0 ? o->etamxf : 0.3;
    cp.etamin = o->etamin > 0 ? o->etamin : 0.1;
    cp.hmin = o->hmin;
    cp.hmax = o->hmax;
    cp.p = p;
    cp.pid_sign_mode = o->pid_sign_mode;
    cp.small_nef = o->small_nef > 0 ? o->small_nef : 2;
    cp.max_nef = o->max_nef > 0 ? o->max_nef : 7;
    return cp;
}

// Fresh controllers for a call; with `keep`, the step proposal and error history of the
// previous call (or of rtbte_set_controller) carry over.
void ctl_reset_all(rtbte_ctx *ctx, double t0, double t_out, long long max_steps, bool keep = false) {
    for (int i = 0; i < n_inst(ctx); ++i) {
        Ctl *c = ctx->ctl_host + i;
        const Ctl prev = *c;
        std::memset(c, 0, sizeof(Ctl));
        c->cur = prev.cur;
        c->t = t0;
        c->t_out = t_out;
        c->eps1 = c->eps2 = 1.0;
        c->first = 1;
        c->max_steps = max_steps;
        if (keep) {
            c->h = prev.h;
            c->eps1 = prev.eps1;
            c->eps2 = prev.eps2;
            c->first = prev.first;
            c->nef = prev.nef;
        }
    }
}

bool can_resume(rtbte_ctx *ctx) {
    for (int i = 0; i < n_inst(ctx); ++i)
        if (!(ctx->ctl_host[i].h > 0)) return false;
    return true;
}

// Fixed-step RK4 of `parts` over [t0, t1] with nominal step h (last step ends at t1), every
// instance in lock step.  Keeps each instance's current buffer.
int fixed_rk4(rtbte_ctx *ctx, const rtbte_integ *o, unsigned parts, double t0, double t1, double h,
              long long *attempts) {
    int rc;
    if ((rc = read_ctl(ctx))) return rc;
    long long nsteps = (long long)ceil((t1 - t0) / h - 1e-9);
    if (nsteps < 1) nsteps = 1;
    ctl_reset_all(ctx, t0, t1, nsteps);
    for (int i = 0; i < n_inst(ctx); ++i) {
        Ctl *c = ctx->ctl_host + i;
        c->fixed = 1;
        c->h = h;
        c->last = nsteps == 1;
        c->h_try = c->last ? t1 - t0 : h;
    }
    if ((rc = write_ctl(ctx))) return rc;
    CtlParams cp = ctl_params(o, 4);
    return run_attempts(ctx, RTBTE_RK4, cp, parts, nullptr, o->chunk > 0 ? o->chunk : kLoopCap, attempts);
}

// Aggregate per-instance controller counters into the call's statistics.
void gather_stats(rtbte_ctx *ctx, rtbte_stats *st, bool add_steps) {
    long long steps = 0, fails = 0;
    double t = 1e300;
    int status = RTBTE_OK;
    for (int i = 0; i < n_inst(ctx); ++i) {
        const Ctl &c = ctx->ctl_host[i];
        steps += c.steps;
        fails += c.fails;
        if (c.t < t) t = c.t;
        if (status == RTBTE_OK && c.status != RTBTE_OK) status = c.status;
    }
    long long rv = 0;
    for (int i = 0; i < n_inst(ctx); ++i) rv += ctx->ctl_host[i].range_viol;
    st->range_violations = add_steps ? st->range_violations + rv : rv;
    st->steps = add_steps ? st->steps + steps : steps;
    st->fails += fails;
    st->t = t;
    st->h_last = ctx->ctl_host[0].h_last;
    st->h_next = ctx->ctl_host[0].h;
    st->status = status;
}

}  // namespace

// The stage kernel's grid is the number of its blocks resident on the whole GPU: a larger
// grid leaves a second partial wave of blocks (at 80 registers, 3 blocks of 256 threads fit an
// SM, so 512 blocks ran as 456 + 56 and the SMs holding the second wave took 1.7x the mean).
int init_stage_grid(rtbte_ctx *ctx) {
    int nb = 0;
    if (ctx->precision == RTBTE_PREC_FP64)
        RT_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage_kernel<double>, kRedThreads, 0));
    else
        RT_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage_kernel<float>, kRedThreads, 0));
    ctx->stage_resident = std::max(nb, 1) * ctx->num_sms;
    return RTBTE_OK;
}


int advance_to(rtbte_ctx *ctx, double t_out, double *y, const rtbte_integ *o, rtbte_stats *st) {
    rtbte_stats local;
    if (!st) st = &local;
    std::memset(st, 0, sizeof(*st));
    const int m = o->method;
    if (m < RTBTE_RK4 || m > RTBTE_MRI_ADAPT) return fail(ctx, RTBTE_E_INVALID_ARG, "unknown method");
    if (!(t_out > o->t0)) return fail(ctx, RTBTE_E_INVALID_ARG, "t_out must exceed t0");
    if ((m == RTBTE_RK4 || m == RTBTE_SPLIT_RK4) && !(o->h > 0)) return fail(ctx, RTBTE_E_INVALID_ARG, "h must be > 0");
    if ((m == RTBTE_MRI_KW3 || m == RTBTE_SPLIT_RK4 || m == RTBTE_MRI_ADAPT) && !(o->h_s > 0))
        return fail(ctx, RTBTE_E_INVALID_ARG, "h_s must be > 0");
    if (m == RTBTE_MRI_ADAPT && (o->fast_tol_scale < 0 || o->slow_safety < 0 || o->slow_fac_min < 0 ||
                                 o->slow_fac_max < 0 || o->slow_max_fail < 0 || !(o->fast_tol_scale <= 1)))
        return fail(ctx, RTBTE_E_INVALID_ARG, "slow-step options must be >= 0 (fast_tol_scale <= 1)");
    if ((m == RTBTE_BS32 || m == RTBTE_ZON43 || m == RTBTE_MRI_KW3 || m == RTBTE_MRI_ADAPT) &&
        (!(o->rtol >= 0) || !(o->atol_c > 0) || !(o->atol_ph > 0)))
        return fail(ctx, RTBTE_E_INVALID_ARG, "tolerances must be positive");
    const size_t nb = sizeof(double) * ctx->n_y;
    RT_CUDA(ctx, cudaMemcpyAsync(ctx->Y[0].p, y, nb, cudaMemcpyDeviceToDevice, ctx->stream));
    const int NI = n_inst(ctx);
    for (int i = 0; i < NI; ++i) ctx->ctl_host[i].cur = 0;
    const long long max_steps = o->max_steps > 0 ? o->max_steps : 1000000000LL;
    const bool resume = o->resume != 0 && can_resume(ctx);
    ctl_reset_all(ctx, o->t0, t_out, max_steps, resume);
    int rc = RTBTE_OK;
    if (m == RTBTE_RK4) {
        if ((rc = write_ctl(ctx))) return rc;
        long long att = 0;
        if ((rc = fixed_rk4(ctx, o, RTBTE_ALL, o->t0, t_out, o->h, &att))) return rc;
        st->attempts = att;
        st->rhs_full = 4 * att;
        gather_stats(ctx, st, false);
    } else if (m == RTBTE_BS32 || m == RTBTE_ZON43) {
        const Tableau T = tableau_of(m);
        CtlParams cp = ctl_params(o, T.p);
        const bool est = !resume && !(o->h0 > 0);
        if (!est && !resume)
            for (int i = 0; i < NI; ++i) ctx->ctl_host[i].h = o->hmax > 0 && o->h0 > o->hmax ? o->hmax : o->h0;
        if ((rc = write_ctl(ctx))) return rc;
        if (est) {
            if ((rc = h0_estimate(ctx, cp, RTBTE_ALL, nullptr, t_out - o->t0))) return rc;
        } else {
            arm_kernel<<<(NI + 127) / 128, 128, 0, ctx->stream>>>(ctx->ctl.as<Ctl>(), NI);
            RT_CUDA(ctx, cudaGetLastError());
            ctx->launches++;
        }
        long long att = 0;
        if ((rc = run_attempts(ctx, m, cp, RTBTE_ALL, nullptr, o->chunk > 0 ? o->chunk : kLoopCap, &att))) return rc;
        st->attempts = att;
        st->rhs_full = att * T.S + (est ? 2LL * NI : 0);
        gather_stats(ctx, st, false);
    } else if (m == RTBTE_MRI_KW3 || m == RTBTE_MRI_ADAPT) {
        const bool adapt = m == RTBTE_MRI_ADAPT;
        const Mis M = mis_kw3();
        const int fm = o->fast_method == RTBTE_BS32 ? RTBTE_BS32 : RTBTE_ZON43;
        const Tableau Tf = tableau_of(fm);
        CtlParams cp = ctl_params(o, Tf.p);
        const CtlParams cps = cp;  // tolerances of the slow-step error norm (adaptive slow step)
        if (adapt) {               // the fast solves run below the slow tolerance
            const double fts = o->fast_tol_scale > 0 ? o->fast_tol_scale : 0.1;
            cp.rtol *= fts;
            cp.atol_c *= fts;
            cp.atol_ph *= fts;
        }
        if (!resume)
            for (int i = 0; i < NI; ++i) ctx->ctl_host[i].h = 0.0;
        if ((rc = write_ctl(ctx))) return rc;
        const long long n = ctx->n_y;
        double *Fs = ctx->Fs.as<double>();
        double *r = ctx->forcing.as<double>();
        const int nb2 = row_grid(ctx);
        long long nsteps = (long long)ceil((t_out - o->t0) / o->h_s - 1e-9);
        if (nsteps < 1) nsteps = 1;
        double t = o->t0;
        bool first_inner = !resume, failed = false;
        long long inner_attempts = 0, inner_h0 = 0;
        StageArgs a = stage_args(ctx, Tf, cp, RTBTE_SLOW, nullptr);
        a.stage = -1;
        a.respect_done = 0;
        // surrogate slow part (single instance): control variate about the last exact value,
        // exact judge every sur_period slow steps, exact for the rest of the call once a judge fails
        bool sur_on = ctx->sur != nullptr && NI == 1 && !adapt;
        st->judge_err_max = -1.0;
        if (sur_on) {  // surrogate values write the sub-lattice rows only; the slow part is 0 elsewhere
            sur_reset(ctx);
            RT_CUDA(ctx, cudaMemsetAsync(Fs, 0, sizeof(double) * 3 * n, ctx->stream));
        }
        auto slow_exact = [&](double *dst) -> int {
            int r2;
            if ((r2 = stage(ctx, a, ctx->stream))) return r2;
            if ((r2 = launch_rhs_core(ctx, RTBTE_SLOW, nullptr, ctx->stream))) return r2;
            if ((r2 = launch_rows(ctx, RTBTE_SLOW, dst, nullptr, ctx->stream))) return r2;
            st->rhs_slow += NI;
            st->slow_exact += NI;
            return RTBTE_OK;
        };
        auto ycur = [&]() { return ctx->Y[ctx->ctl_host[0].cur].as<double>(); };
        // MIS stages 2..4 of one slow step from t over H (Fs holds the slow value at z_1 = y):
        // constant forcing per stage, inner adaptive ERK over the stage's sub-interval
        auto mis_stages = [&](double t, double H) -> int {
            for (int i = 1; i <= 3; ++i) {
                const double dc = M.chat[i] - M.chat[i - 1];
                const double ta = t + M.chat[i - 1] * H, tb = (i == 3) ? t + H : t + M.chat[i] * H;
                mri_forcing<<<nb2, kRedThreads, 0, ctx->stream>>>(r, Fs, M.Om[i][0], M.Om[i][1], M.Om[i][2], i, dc, n);
                mri_stage_reset<<<(NI + 127) / 128, 128, 0, ctx->stream>>>(ctx->ctl.as<Ctl>(), NI, cp, ta, tb);
                RT_CUDA(ctx, cudaGetLastError());
                ctx->launches += 2;
                if (first_inner) {
                    if ((rc = h0_estimate(ctx, cp, RTBTE_FAST, r, tb - ta))) return rc;
                    inner_h0++;
                    first_inner = false;
                }
                long long att = 0;
                if ((rc = run_attempts(ctx, fm, cp, RTBTE_FAST, r, o->chunk > 0 ? o->chunk : kLoopCap, &att))) return rc;
                inner_attempts += att;
                for (int q = 0; q < NI; ++q)
                    if (ctx->ctl_host[q].status != RTBTE_OK) failed = true;
                if (failed) break;
                if (i < 3) {
                    if (sur_on) {
                        if ((rc = sur_value(ctx, ycur(), Fs + (long long)i * n))) return rc;
                        st->slow_surrogate++;
                    } else if ((rc = slow_exact(Fs + (long long)i * n))) {
                        return rc;
                    }
                }
            }
            return RTBTE_OK;
        };
        int slow_status = RTBTE_OK;
        if (!adapt) {
            for (long long k = 0; k < nsteps && !failed; ++k) {
                const double H = (k == nsteps - 1) ? t_out - t : o->h_s;
                // slow RHS at z_1 = y
                if (!sur_on || k % ctx->sur_period == 0) {
                    if ((rc = slow_exact(Fs))) return rc;
                    if (sur_on) {
                        double e = 0;
                        if ((rc = sur_judge(ctx, ycur(), Fs, &e))) return rc;
                        st->judge_err_max = std::max(st->judge_err_max, e);
                        if (e > ctx->sur_tol) {
                            sur_on = false;
                            st->surrogate_fallbacks = 1;
                        }
                    }
                } else {
                    if ((rc = sur_value(ctx, ycur(), Fs))) return rc;
                    st->slow_surrogate++;
                }
                if ((rc = mis_stages(t, H))) return rc;
                if (failed) break;
                t = (k == nsteps - 1) ? t_out : t + H;
                st->slow_steps++;
            }
        } else {
            // slow step from the tolerance by step doubling: one MIS step of Hk and two of Hk/2
            // from y_n, local error of the latter (y_1 - y_2) / (2^3 - 1) in the WRMS norm of the
            // slow tolerances with weights from y_n; the largest norm over instances decides
            const double safety = o->slow_safety > 0 ? o->slow_safety : 0.9;
            const double fac_min = o->slow_fac_min > 0 ? o->slow_fac_min : 0.2;
            const double fac_max = o->slow_fac_max > 0 ? o->slow_fac_max : 5.0;
            const int max_fail = o->slow_max_fail > 0 ? o->slow_max_fail : 7;
            const size_t need = sizeof(double) * (2 * (size_t)n + (size_t)NI);
            if (ctx->slow_save.bytes < need) {
                ctx->slow_save.release();
                RT_CUDA(ctx, cudaMalloc(&ctx->slow_save.p, need));
                ctx->slow_save.bytes = need;
            }
            double *yn = ctx->slow_save.as<double>(), *y1 = yn + n, *eps_d = y1 + n;
            double *Y0 = ctx->Y[0].as<double>(), *Y1 = ctx->Y[1].as<double>();
            Ctl *cd = ctx->ctl.as<Ctl>();
            const RowParams Q = row_params(ctx);
            double *wsq = ctx->wrms_part.as<double>(), *part = wsq + 2 * n;
            std::vector<double> h_in0(NI), eps_h(NI);
            double H = resume && ctx->h_slow > 0 ? ctx->h_slow : o->h_s;
            int nfail = 0;
            bool after_fail = false;
            auto copy = [&](double *buf, int to_buf) -> int {
                copy_cur<<<nb2, kRedThreads, 0, ctx->stream>>>(Q, cd, Y0, Y1, buf, n, to_buf);
                RT_CUDA(ctx, cudaGetLastError());
                ctx->launches++;
                return RTBTE_OK;
            };
            // back to y_n and the fast step proposals held there (the mirror is current: every
            // fast solve ends with a controller read-back)
            auto restore = [&](bool first0) -> int {
                int r2;
                if ((r2 = copy(yn, 0))) return r2;
                for (int q = 0; q < NI; ++q) ctx->ctl_host[q].h = h_in0[q];
                if ((r2 = write_ctl(ctx))) return r2;
                first_inner = first0;
                return RTBTE_OK;
            };
            while (t < t_out) {
                if (st->slow_steps >= max_steps) {
                    slow_status = RTBTE_E_TOO_MANY_STEPS;
                    break;
                }
                double Hk = H;
                bool last = false;
                if (t + Hk >= t_out) {
                    Hk = t_out - t;
                    last = true;
                }
                if ((rc = copy(yn, 1))) return rc;
                for (int q = 0; q < NI; ++q) h_in0[q] = ctx->ctl_host[q].h;
                const bool first0 = first_inner;
                // one step of Hk
                if ((rc = slow_exact(Fs)) || (rc = mis_stages(t, Hk))) return rc;
                if (failed) {
                    if ((rc = restore(first0))) return rc;
                    break;
                }
                if ((rc = copy(y1, 1)) || (rc = restore(first0))) return rc;
                // two steps of Hk / 2
                const double Hh = 0.5 * Hk, tm = t + Hh;
                if ((rc = slow_exact(Fs)) || (rc = mis_stages(t, Hh))) return rc;
                if (!failed && ((rc = slow_exact(Fs)) || (rc = mis_stages(tm, Hh)))) return rc;
                if (failed) {
                    if ((rc = restore(first0))) return rc;
                    break;
                }
                slow_err_sq<<<nb2, kRedThreads, 0, ctx->stream>>>(Q, cps, cd, Y0, Y1, yn, y1, wsq, n);
                wrms_chunks<<<dim3(kWrmsChunks, NI), kRedThreads, 0, ctx->stream>>>(Q, cd, wsq, part, 0);
                slow_eps<<<NI, kRedThreads, 0, ctx->stream>>>(Q, part, eps_d);
                RT_CUDA(ctx, cudaGetLastError());
                ctx->launches += 3;
                RT_CUDA(ctx, cudaMemcpyAsync(eps_h.data(), eps_d, sizeof(double) * NI, cudaMemcpyDeviceToHost,
                                             ctx->stream));
                RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
                double eps = 0.0;
                bool finite = true;
                for (double e : eps_h) {
                    if (!std::isfinite(e)) finite = false;
                    else eps = std::max(eps, e);
                }
                if (!finite) {
                    slow_status = RTBTE_E_NONFINITE;
                    if ((rc = restore(first0))) return rc;
                    break;
                }
                if (eps <= 1.0) {  // accept y_2; the fast proposal continues from the second half step
                    t = last ? t_out : t + Hk;
                    st->slow_steps++;
                    double fac = safety * std::pow(std::max(eps, 1e-10), -0.25);
                    fac = std::min(fac, after_fail ? 1.0 : fac_max);
                    fac = std::max(fac, fac_min);
                    H = Hk * fac;
                    nfail = 0;
                    after_fail = false;
                } else {
                    if ((rc = restore(first0))) return rc;
                    st->slow_fails++;
                    if (++nfail >= max_fail) {
                        slow_status = RTBTE_E_ERR_TEST_FAIL;
                        break;
                    }
                    double fac = std::min(safety * std::pow(eps, -0.25), 1.0);
                    fac = std::max(fac, fac_min);
                    H = Hk * fac;
                    after_fail = true;
                }
                if (t < t_out && !(t + H > t)) {
                    slow_status = RTBTE_E_STEP_UNDERFLOW;
                    break;
                }
            }
            ctx->h_slow = H;
            st->h_slow_next = H;
        }
        st->attempts = inner_attempts;
        st->rhs_fast = inner_attempts * Tf.S + 2LL * NI * inner_h0;
        gather_stats(ctx, st, false);
        if (!failed || adapt) st->t = t;
        if (st->status == RTBTE_OK) st->status = slow_status;
    } else {  // first-order operator splitting with RK4 (slow step, then fast sub-steps)
        if ((rc = write_ctl(ctx))) return rc;
        long long nsteps = (long long)ceil((t_out - o->t0) / o->h_s - 1e-9);
        if (nsteps < 1) nsteps = 1;
        double t = o->t0;
        long long att_s = 0, att_f = 0;
        bool failed = false;
        for (long long k = 0; k < nsteps && !failed; ++k) {
            const double H = (k == nsteps - 1) ? t_out - t : o->h_s;
            long long a1 = 0, a2 = 0;
            if ((rc = fixed_rk4(ctx, o, RTBTE_SLOW, t, t + H, H, &a1))) return rc;
            att_s += a1;
            for (int q = 0; q < NI; ++q)
                if (ctx->ctl_host[q].status != RTBTE_OK) failed = true;
            if (failed) break;
            long long msub = (long long)floor(H / o->h + 0.5);
            if (msub < 1) msub = 1;
            if ((rc = fixed_rk4(ctx, o, RTBTE_FAST, t, t + H, H / (double)msub, &a2))) return rc;
            att_f += a2;
            gather_stats(ctx, st, true);
            for (int q = 0; q < NI; ++q)
                if (ctx->ctl_host[q].status != RTBTE_OK) failed = true;
            if (failed) break;
            t = (k == nsteps - 1) ? t_out : t + H;
            st->slow_steps++;
        }
        st->attempts = att_s + att_f;
        st->rhs_slow = 4 * att_s;
        st->rhs_fast = 4 * att_f;
        const long long steps = st->steps;
        gather_stats(ctx, st, false);
        st->steps = steps;
        if (!failed) st->t = t;
    }
    // hand back each instance's current buffer (the solution, or its last accepted state)
    for (int i = 0; i < NI; ++i) {
        const InstHost &I = ctx->inst[i];
        const size_t off = (size_t)I.y_off, cnt = (size_t)(I.d.n_c + I.n_ph);
        RT_CUDA(ctx, cudaMemcpyAsync(y + off, ctx->Y[ctx->ctl_host[i].cur].as<double>() + off, sizeof(double) * cnt,
                                     cudaMemcpyDeviceToDevice, ctx->stream));
    }
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (st->status) fail(ctx, st->status, "integration stopped before t_out");
    return st->status;
}

void destroy_graphs(rtbte_ctx *ctx) {
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    ctx->graphs.clear();
    ctx->graph_launches.clear();
}

}  // namespace rtbte
