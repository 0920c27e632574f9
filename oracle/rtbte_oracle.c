/*
 * rtbte_oracle.c -- plain FP64 CPU oracle for the coupled electron/phonon
 * real-time Boltzmann equation (rt-BTE) and its time integrators.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; it is used by tests/, by __graft_entry__.smoke() and by bench.py's CPU
 * baseline leg.  It shares no code, header, table or constant with the CUDA
 * library: every formula below is written out again from the paper.
 *
 * What it computes (paper sections cited per function):
 *   - the scattering-channel lists that are "computed and stored before the
 *     real-time simulation" (Results, Sec. rt-BTE), by brute-force enumeration;
 *   - the collision integrals I^{e-ph}, I^{ph-e} (Eq. e-ph with the F_em/F_abs
 *     factors) and I^{ph-ph} (Eq. ph-ph with G_em/G_abs), both directly from the
 *     definition (no list) and from the stored lists;
 *   - fixed-step RK4, adaptive ERK with the embedded error estimate
 *     (Eq. ERK_method), the WRMS norm (Eqs. wrms_norm, wrms_weights), the PID
 *     step controller (Eq. pid_controller), and the explicit MRI/MIS algorithm
 *     (Methods B, Eq. mis_coef), plus first-order RK4 operator splitting.
 *
 * Readings where the paper is silent or garbled:
 *   - Gaussian delta: exp(-(E/sigma)^2)/(sigma*sqrt(pi)), truncated at |E|>3 sigma
 *     (the printed form in Methods A is not normalisable).
 *   - MIS last-stage coupling uses b_j - A_{S,j} (the printed A_{S-1,j} breaks
 *     the reduction of MIS to its base ERK method when the fast part vanishes).
 *   - PID exponents alternate in sign (-a1, +a2, -a3), ARKODE's documented form;
 *     the all-negative printed form is selectable.
 *   - Controller constants not in the paper follow ARKODE's documented defaults.
 *   - The slow step of the tolerance-chosen MRI (future work in the Discussion) is
 *     controlled by step doubling with library constants (or_mri_adapt_solve).
 *
 * Parity pins: see tests/test_oracle_*.py (detailed balance, conservation laws,
 * brute force, closed-form ODE solutions, order conditions).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ---------------------------------------------------------------------------
 * Model description (filled from Python; the arrays come from rtbte_inputs)
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t dim, fold, nbands, nmodes;
    int32_t nk[3];
    int32_t nq[3];
    int32_t n_c, pp_stride, lut_bits, pad0;
    const int32_t *e_band;  /* [n_c] */
    const int32_t *e_k;     /* [n_c*3] */
    const double *e_eps;    /* [n_c] eV */
    const double *ph_omega; /* [nmodes*N_q] hbar*omega, eV */
    const double *g2_coef;  /* [nmodes] median |g|^2 per mode, eV^2 */
    const double *lut;      /* [2^lut_bits] lognormal shape factors */
    double v3_coef;         /* median |V3|^2 */
    double sigma_eph, sigma_pp, omega_cut, hbar;
    uint64_t g2_seed, v3_seed;
} or_model;

/* Stored channel lists (CSR).  e-ph: 2 sub-segments per electron destination
 * (emission then absorption), each ordered by (mode, source state).  ph-e: one
 * segment per phonon, ordered by (electron destination, electron source).
 * ph-ph: 2 sub-segments per sub-lattice phonon (emission pairs b<=c, then
 * absorption), ordered by (b, c). */

static long prod3(const int32_t *n) { return (long)n[0] * n[1] * n[2]; }

static int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

static int min_image(int d, int n) {
    d = wrap(d, n);
    if (d > n / 2) d -= n;
    return d;
}

static long klin(const int32_t *n, int x, int y, int z) { return ((long)z * n[1] + y) * n[0] + x; }

/* SplitMix64 output function (Steele, Lea & Flood 2014), used as a keyed hash. */
static uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double lut_draw(const or_model *m, uint64_t seed, uint64_t key) {
    uint64_t h = mix64(key ^ mix64(seed));
    return m->lut[h >> (64 - m->lut_bits)];
}

/* Gaussian approximation of the energy delta (Methods A; normalised reading). */
static double gauss_delta(double E, double sigma) {
    double x = E / sigma;
    return exp(-x * x) / (sigma * sqrt(OR_PI));
}

/* ---- electron-state helpers ---------------------------------------------- */
typedef struct {
    long Nk, Nq, Nph;
    int *kmap;        /* [nbands*Nk] windowed index or -1 */
} or_aux;

static void aux_init(const or_model *m, or_aux *a) {
    a->Nk = prod3(m->nk);
    a->Nq = prod3(m->nq);
    a->Nph = (long)m->nmodes * a->Nq;
    a->kmap = (int *)malloc(sizeof(int) * (size_t)m->nbands * (size_t)a->Nk);
    for (long i = 0; i < (long)m->nbands * a->Nk; ++i) a->kmap[i] = -1;
    for (int s = 0; s < m->n_c; ++s) {
        const int32_t *k = m->e_k + 3 * s;
        a->kmap[(long)m->e_band[s] * a->Nk + klin(m->nk, k[0], k[1], k[2])] = s;
    }
}

static void aux_free(or_aux *a) { free(a->kmap); }

/* Phonon wave vector linking electron k (dest) to k' (src): q = T(k' - k), the
 * min-image difference on the electron grid mapped to the phonon grid by
 * truncating division by the grid ratio. */
static long q_of(const or_model *m, const int32_t *kd, const int32_t *ks) {
    int q[3];
    for (int c = 0; c < 3; ++c) {
        int d = min_image(ks[c] - kd[c], m->nk[c]);
        q[c] = wrap(d / m->fold, m->nq[c]);
    }
    return klin(m->nq, q[0], q[1], q[2]);
}

static uint64_t e_state_id(const or_model *m, long Nk, int s) {
    const int32_t *k = m->e_k + 3 * s;
    return (uint64_t)m->e_band[s] * (uint64_t)Nk + (uint64_t)klin(m->nk, k[0], k[1], k[2]);
}

static uint64_t e_state_id_inv(const or_model *m, long Nk, int s) {
    const int32_t *k = m->e_k + 3 * s;
    return (uint64_t)m->e_band[s] * (uint64_t)Nk +
           (uint64_t)klin(m->nk, wrap(-k[0], m->nk[0]), wrap(-k[1], m->nk[1]), wrap(-k[2], m->nk[2]));
}

/* |g_{mn nu}|^2 for the process linking electron states s1, s2 via mode nu:
 * symmetric in (s1, s2) and under inversion (k -> -k). */
static double g2_of(const or_model *m, long Nk, int s1, int s2, int nu) {
    uint64_t u1 = e_state_id(m, Nk, s1), u2 = e_state_id(m, Nk, s2);
    uint64_t v1 = e_state_id_inv(m, Nk, s1), v2 = e_state_id_inv(m, Nk, s2);
    uint64_t lo = u1 < u2 ? u1 : u2, hi = u1 < u2 ? u2 : u1;
    uint64_t ilo = v1 < v2 ? v1 : v2, ihi = v1 < v2 ? v2 : v1;
    if (ilo < lo || (ilo == lo && ihi < hi)) { lo = ilo; hi = ihi; }
    uint64_t U = (uint64_t)m->nbands * (uint64_t)Nk;
    uint64_t key = (lo * U + hi) * (uint64_t)m->nmodes + (uint64_t)nu;
    return m->g2_coef[nu] * lut_draw(m, m->g2_seed, key);
}

/* e-ph weight: (2 pi / hbar)(1/N_q) |g|^2 delta(Delta)  (Eq. e-ph). */
static double w_eph(const or_model *m, const or_aux *a, int d, int s, int nu, double Delta) {
    double pref = 2.0 * OR_PI / m->hbar / (double)a->Nq;
    return pref * g2_of(m, a->Nk, d, s, nu) * gauss_delta(Delta, m->sigma_eph);
}

/* ph-e weight: (4 pi / hbar)(1/N_k) |g|^2 delta(Delta)  (Eq. e-ph, second line). */
static double w_phe(const or_model *m, const or_aux *a, int d, int s, int nu, double Delta) {
    double pref = 4.0 * OR_PI / m->hbar / (double)a->Nk;
    return pref * g2_of(m, a->Nk, d, s, nu) * gauss_delta(Delta, m->sigma_eph);
}

/* Channel predicate for e-ph destination d, source s, phonon p.
 * proc 0 = emission:   Delta = (eps_d - hw_p) - eps_s   (Eq. e-ph, first delta)
 * proc 1 = absorption: Delta = (eps_s - hw_p) - eps_d   (the negated second delta)
 * Both are written as (eps_hi - hw) - eps_lo with the emitting state first, so the
 * emission entry (d <- s) and its absorption partner (s <- d) see the same bits. */
static int eph_keep(const or_model *m, int d, int s, long p, int proc, double *Delta) {
    double w = m->ph_omega[p];
    if (w < m->omega_cut) return 0;
    double D = proc == 0 ? (m->e_eps[d] - w) - m->e_eps[s] : (m->e_eps[s] - w) - m->e_eps[d];
    double cut = 3.0 * m->sigma_eph;
    *Delta = D;
    return D <= cut && D >= -cut;
}

/* ---------------------------------------------------------------------------
 * e-ph channel list (destination-sorted)
 * ------------------------------------------------------------------------- */
static long eph_dest(const or_model *m, const or_aux *a, int d, int proc, int32_t *src, int32_t *ph,
                     double *W) {
    long cnt = 0;
    const int32_t *kd = m->e_k + 3 * d;
    for (int nu = 0; nu < m->nmodes; ++nu) {
        for (int s = 0; s < m->n_c; ++s) {
            long p = (long)nu * a->Nq + q_of(m, kd, m->e_k + 3 * s);
            double D;
            if (!eph_keep(m, d, s, p, proc, &D)) continue;
            if (src) {
                src[cnt] = s;
                ph[cnt] = (int32_t)p;
                W[cnt] = w_eph(m, a, d, s, nu, D);
            }
            ++cnt;
        }
    }
    return cnt;
}

/* counts[2*i+proc] for the i-th listed destination (dests==NULL: all). */
void or_eph_count(const or_model *m, int ndest, const int32_t *dests, int64_t *counts) {
    or_aux a;
    aux_init(m, &a);
    int n = dests ? ndest : m->n_c;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < n; ++i) {
        int d = dests ? dests[i] : i;
        counts[2 * i] = eph_dest(m, &a, d, 0, NULL, NULL, NULL);
        counts[2 * i + 1] = eph_dest(m, &a, d, 1, NULL, NULL, NULL);
    }
    aux_free(&a);
}

/* off has 2*n+1 entries (exclusive prefix of counts). */
void or_eph_fill(const or_model *m, int ndest, const int32_t *dests, const int64_t *off, int32_t *src,
                 int32_t *ph, double *W) {
    or_aux a;
    aux_init(m, &a);
    int n = dests ? ndest : m->n_c;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < n; ++i) {
        int d = dests ? dests[i] : i;
        for (int proc = 0; proc < 2; ++proc) {
            long o = off[2 * i + proc];
            eph_dest(m, &a, d, proc, src + o, ph + o, W + o);
        }
    }
    aux_free(&a);
}

/* ---------------------------------------------------------------------------
 * ph-e channel list (phonon-sorted absorption processes)
 * ------------------------------------------------------------------------- */
static int cmp_int(const void *x, const void *y) {
    int a = *(const int *)x, b = *(const int *)y;
    return (a > b) - (a < b);
}

/* Electron sources s with T(k_s - k_d) = q, in ascending order. */
static int phe_sources(const or_model *m, const or_aux *a, int d, const int *qc, int *out) {
    const int32_t *kd = m->e_k + 3 * d;
    int pre[3][8], npre[3];
    for (int c = 0; c < 3; ++c) {
        npre[c] = 0;
        int n = m->nk[c];
        for (int dd = -(n - 1) / 2; dd <= n / 2; ++dd) {
            if (wrap(dd / m->fold, m->nq[c]) == qc[c]) pre[c][npre[c]++] = dd;
        }
    }
    int cnt = 0;
    for (int i0 = 0; i0 < npre[0]; ++i0)
        for (int i1 = 0; i1 < npre[1]; ++i1)
            for (int i2 = 0; i2 < npre[2]; ++i2) {
                long kl = klin(m->nk, wrap(kd[0] + pre[0][i0], m->nk[0]), wrap(kd[1] + pre[1][i1], m->nk[1]),
                               wrap(kd[2] + pre[2][i2], m->nk[2]));
                for (int b = 0; b < m->nbands; ++b) {
                    int s = a->kmap[(long)b * a->Nk + kl];
                    if (s >= 0) out[cnt++] = s;
                }
            }
    qsort(out, cnt, sizeof(int), cmp_int);
    return cnt;
}

static void q_coords(const or_model *m, long ql, int *qc) {
    qc[0] = (int)(ql % m->nq[0]);
    qc[1] = (int)((ql / m->nq[0]) % m->nq[1]);
    qc[2] = (int)(ql / ((long)m->nq[0] * m->nq[1]));
}

static long phe_phonon(const or_model *m, const or_aux *a, long p, int32_t *dst, int32_t *src, double *W) {
    if (m->ph_omega[p] < m->omega_cut) return 0;
    int nu = (int)(p / a->Nq);
    int qc[3];
    q_coords(m, p % a->Nq, qc);
    int cand[512]; /* up to 3 preimages per dimension times nbands (<= 16) */
    long cnt = 0;
    for (int d = 0; d < m->n_c; ++d) {
        int nc = phe_sources(m, a, d, qc, cand);
        for (int j = 0; j < nc; ++j) {
            int s = cand[j];
            double D;
            if (!eph_keep(m, d, s, p, 1, &D)) continue;
            if (dst) {
                dst[cnt] = d;
                src[cnt] = s;
                W[cnt] = w_phe(m, a, d, s, nu, D);
            }
            ++cnt;
        }
    }
    return cnt;
}

void or_phe_count(const or_model *m, int nph, const int64_t *phs, int64_t *counts) {
    or_aux a;
    aux_init(m, &a);
    long n = phs ? nph : a.Nph;
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < n; ++i) counts[i] = phe_phonon(m, &a, phs ? phs[i] : i, NULL, NULL, NULL);
    aux_free(&a);
}

void or_phe_fill(const or_model *m, int nph, const int64_t *phs, const int64_t *off, int32_t *dst,
                 int32_t *src, double *W) {
    or_aux a;
    aux_init(m, &a);
    long n = phs ? nph : a.Nph;
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < n; ++i) {
        long o = off[i];
        phe_phonon(m, &a, phs ? phs[i] : i, dst + o, src + o, W + o);
    }
    aux_free(&a);
}

/* ---------------------------------------------------------------------------
 * ph-ph channel list on the stride-s sub-lattice
 * ------------------------------------------------------------------------- */
typedef struct {
    int nqs[3];
    long Nqs, M;
    long *full;  /* [M] full phonon index of each sub-lattice state */
} or_pp;

static void pp_init(const or_model *m, const or_aux *a, or_pp *pp) {
    int st = m->pp_stride;
    for (int c = 0; c < 3; ++c) pp->nqs[c] = m->nq[c] > 1 ? m->nq[c] / st : 1;
    pp->Nqs = (long)pp->nqs[0] * pp->nqs[1] * pp->nqs[2];
    pp->M = (long)m->nmodes * pp->Nqs;
    pp->full = (long *)malloc(sizeof(long) * (size_t)pp->M);
    for (int nu = 0; nu < m->nmodes; ++nu)
        for (long ql = 0; ql < pp->Nqs; ++ql) {
            int x = (int)(ql % pp->nqs[0]), y = (int)((ql / pp->nqs[0]) % pp->nqs[1]),
                z = (int)(ql / ((long)pp->nqs[0] * pp->nqs[1]));
            int sx = m->nq[0] > 1 ? st : 1, sy = m->nq[1] > 1 ? st : 1, sz = m->nq[2] > 1 ? st : 1;
            pp->full[(long)nu * pp->Nqs + ql] = (long)nu * a->Nq + klin(m->nq, x * sx, y * sy, z * sz);
        }
}

static long ph_inv(const or_model *m, const or_aux *a, long p) {
    int nu = (int)(p / a->Nq);
    int qc[3];
    q_coords(m, p % a->Nq, qc);
    return (long)nu * a->Nq + klin(m->nq, wrap(-qc[0], m->nq[0]), wrap(-qc[1], m->nq[1]), wrap(-qc[2], m->nq[2]));
}

static void sort3(uint64_t *t) {
    uint64_t x;
    if (t[0] > t[1]) { x = t[0]; t[0] = t[1]; t[1] = x; }
    if (t[1] > t[2]) { x = t[1]; t[1] = t[2]; t[2] = x; }
    if (t[0] > t[1]) { x = t[0]; t[0] = t[1]; t[1] = x; }
}

/* |V3|^2 for the three full phonon states: symmetric in the three and under q -> -q. */
static double v3_of(const or_model *m, const or_aux *a, long p1, long p2, long p3) {
    uint64_t t[3] = {(uint64_t)p1, (uint64_t)p2, (uint64_t)p3};
    uint64_t u[3] = {(uint64_t)ph_inv(m, a, p1), (uint64_t)ph_inv(m, a, p2), (uint64_t)ph_inv(m, a, p3)};
    sort3(t);
    sort3(u);
    if (u[0] < t[0] || (u[0] == t[0] && (u[1] < t[1] || (u[1] == t[1] && u[2] < t[2])))) {
        t[0] = u[0]; t[1] = u[1]; t[2] = u[2];
    }
    uint64_t N = (uint64_t)a->Nph;
    uint64_t key = (t[0] * N + t[1]) * N + t[2];
    return m->v3_coef * lut_draw(m, m->v3_seed, key);
}

/* ph-ph weight (36 pi/hbar)(1/N_q,pp)|V3|^2 delta(Delta)  (Eq. ph-ph). */
static double w_pp(const or_model *m, const or_aux *a, const or_pp *pp, long pa, long pb, long pc, double D) {
    double pref = 36.0 * OR_PI / m->hbar / (double)pp->Nqs;
    return pref * v3_of(m, a, pa, pb, pc) * gauss_delta(D, m->sigma_pp);
}

static long pp_lin(const or_pp *pp, int x, int y, int z) { return ((long)z * pp->nqs[1] + y) * pp->nqs[0] + x; }

static void pp_coords(const or_pp *pp, long ql, int *c) {
    c[0] = (int)(ql % pp->nqs[0]);
    c[1] = (int)((ql / pp->nqs[0]) % pp->nqs[1]);
    c[2] = (int)(ql / ((long)pp->nqs[0] * pp->nqs[1]));
}

/* Enumerate the entries of sub-lattice destination a.
 * proc 0 (emission, a -> b + c, q_c = q_a - q_b): unordered pairs b <= c, weight
 *   doubled when b != c because the ordered sum of Eq. ph-ph counts (b,c) and (c,b).
 * proc 1 (absorption, a + c -> b, q_c = q_b - q_a): weight 2 W (Eq. ph-ph).
 * Delta is (w_lo1 + w_lo2) - w_hi for the process, the same bits at every participant. */
static long pp_dest(const or_model *m, const or_aux *a, const or_pp *pp, long ia, int proc, int32_t *bo,
                    int32_t *co, double *W) {
    long pa = pp->full[ia];
    double wa = m->ph_omega[pa];
    if (wa < m->omega_cut) return 0;
    int qa[3], qb[3];
    pp_coords(pp, ia % pp->Nqs, qa);
    double cut = 3.0 * m->sigma_pp;
    long cnt = 0;
    for (long ib = 0; ib < pp->M; ++ib) {
        long pb = pp->full[ib];
        double wb = m->ph_omega[pb];
        if (wb < m->omega_cut) continue;
        pp_coords(pp, ib % pp->Nqs, qb);
        int sgn = proc == 0 ? 1 : -1;
        long qcl = pp_lin(pp, wrap(sgn * (qa[0] - qb[0]), pp->nqs[0]), wrap(sgn * (qa[1] - qb[1]), pp->nqs[1]),
                          wrap(sgn * (qa[2] - qb[2]), pp->nqs[2]));
        for (int nu2 = 0; nu2 < m->nmodes; ++nu2) {
            long ic = (long)nu2 * pp->Nqs + qcl;
            if (proc == 0 && ic < ib) continue;
            long pc = pp->full[ic];
            double wc = m->ph_omega[pc];
            if (wc < m->omega_cut) continue;
            double D = proc == 0 ? (wb + wc) - wa : (wa + wc) - wb;
            if (!(D <= cut && D >= -cut)) continue;
            if (bo) {
                bo[cnt] = (int32_t)ib;
                co[cnt] = (int32_t)ic;
                double w = w_pp(m, a, pp, pa, pb, pc, D);
                W[cnt] = proc == 0 ? (ib == ic ? w : 2.0 * w) : 2.0 * w;
            }
            ++cnt;
        }
    }
    return cnt;
}

long or_pp_size(const or_model *m) {
    or_aux a;
    aux_init(m, &a);
    or_pp pp;
    pp_init(m, &a, &pp);
    long M = pp.M;
    free(pp.full);
    aux_free(&a);
    return M;
}

void or_pp_full_index(const or_model *m, int64_t *out) {
    or_aux a;
    aux_init(m, &a);
    or_pp pp;
    pp_init(m, &a, &pp);
    for (long i = 0; i < pp.M; ++i) out[i] = pp.full[i];
    free(pp.full);
    aux_free(&a);
}

void or_pp_count(const or_model *m, int ndest, const int64_t *dests, int64_t *counts) {
    or_aux a;
    aux_init(m, &a);
    or_pp pp;
    pp_init(m, &a, &pp);
    long n = dests ? ndest : pp.M;
#pragma omp parallel for schedule(dynamic, 4)
    for (long i = 0; i < n; ++i) {
        long ia = dests ? dests[i] : i;
        counts[2 * i] = pp_dest(m, &a, &pp, ia, 0, NULL, NULL, NULL);
        counts[2 * i + 1] = pp_dest(m, &a, &pp, ia, 1, NULL, NULL, NULL);
    }
    free(pp.full);
    aux_free(&a);
}

void or_pp_fill(const or_model *m, int ndest, const int64_t *dests, const int64_t *off, int32_t *b, int32_t *c,
                double *W) {
    or_aux a;
    aux_init(m, &a);
    or_pp pp;
    pp_init(m, &a, &pp);
    long n = dests ? ndest : pp.M;
#pragma omp parallel for schedule(dynamic, 4)
    for (long i = 0; i < n; ++i) {
        long ia = dests ? dests[i] : i;
        for (int proc = 0; proc < 2; ++proc) {
            long o = off[2 * i + proc];
            pp_dest(m, &a, &pp, ia, proc, b + o, c + o, W + o);
        }
    }
    free(pp.full);
    aux_free(&a);
}

/* ---------------------------------------------------------------------------
 * Population factors, literal forms (Methods A)
 * ------------------------------------------------------------------------- */
static double F_em(double f, double fp, double N) { return f * (1.0 - fp) * (1.0 + N) - (1.0 - f) * fp * N; }
static double F_abs(double f, double fp, double N) { return f * (1.0 - fp) * N - (1.0 - f) * fp * (1.0 + N); }
static double G_em(double N, double N1, double N2) { return N * (N1 + 1.0) * (N2 + 1.0) - (N + 1.0) * N1 * N2; }
static double G_abs(double N, double N1, double N2) { return N * (N1 + 1.0) * N2 - (N + 1.0) * N1 * (N2 + 1.0); }

double or_F_em(double f, double fp, double N) { return F_em(f, fp, N); }
double or_F_abs(double f, double fp, double N) { return F_abs(f, fp, N); }
double or_G_em(double N, double N1, double N2) { return G_em(N, N1, N2); }
double or_G_abs(double N, double N1, double N2) { return G_abs(N, N1, N2); }
double or_gauss_delta(double E, double sigma) { return gauss_delta(E, sigma); }

enum { OR_EPH = 1, OR_PHE = 2, OR_PHPH = 4 };

/* ---------------------------------------------------------------------------
 * RHS directly from the definition (no stored list).  mask selects destinations:
 * emask[n_c] / pmask[N_ph] (NULL = all); unselected outputs are left untouched.
 * ------------------------------------------------------------------------- */
void or_rhs_literal(const or_model *m, const double *y, double *ydot, unsigned parts, const uint8_t *emask,
                    const uint8_t *pmask) {
    or_aux a;
    aux_init(m, &a);
    const double *f = y, *N = y + m->n_c;
    double *df = ydot, *dN = ydot + m->n_c;
    if (parts & OR_EPH) {
        double pref = 2.0 * OR_PI / m->hbar / (double)a.Nq;
#pragma omp parallel for schedule(dynamic, 4)
        for (int d = 0; d < m->n_c; ++d) {
            if (emask && !emask[d]) continue;
            double acc = 0.0;
            const int32_t *kd = m->e_k + 3 * d;
            for (int nu = 0; nu < m->nmodes; ++nu)
                for (int s = 0; s < m->n_c; ++s) {
                    long p = (long)nu * a.Nq + q_of(m, kd, m->e_k + 3 * s);
                    double w = m->ph_omega[p];
                    if (w < m->omega_cut) continue;
                    double g2 = g2_of(m, a.Nk, d, s, nu);
                    double Dem = m->e_eps[d] - w - m->e_eps[s];
                    double Dab = m->e_eps[d] + w - m->e_eps[s];
                    double term = 0.0;
                    if (fabs(Dem) <= 3.0 * m->sigma_eph) term += F_em(f[d], f[s], N[p]) * gauss_delta(Dem, m->sigma_eph);
                    if (fabs(Dab) <= 3.0 * m->sigma_eph) term += F_abs(f[d], f[s], N[p]) * gauss_delta(Dab, m->sigma_eph);
                    acc += g2 * term;
                }
            df[d] = -pref * acc;
        }
    } else {
        for (int d = 0; d < m->n_c; ++d)
            if (!emask || emask[d]) df[d] = 0.0;
    }
    for (long p = 0; p < a.Nph; ++p)
        if (!pmask || pmask[p]) dN[p] = 0.0;
    if (parts & OR_PHE) {
        double pref = 4.0 * OR_PI / m->hbar / (double)a.Nk;
#pragma omp parallel for schedule(dynamic, 16)
        for (long p = 0; p < a.Nph; ++p) {
            if (pmask && !pmask[p]) continue;
            double w = m->ph_omega[p];
            if (w < m->omega_cut) continue;
            int nu = (int)(p / a.Nq);
            int qc[3];
            q_coords(m, p % a.Nq, qc);
            int cand[512];
            double acc = 0.0;
            for (int d = 0; d < m->n_c; ++d) {
                int nc = phe_sources(m, &a, d, qc, cand);
                for (int j = 0; j < nc; ++j) {
                    int s = cand[j];
                    double Dab = m->e_eps[d] + w - m->e_eps[s];
                    if (fabs(Dab) > 3.0 * m->sigma_eph) continue;
                    acc += g2_of(m, a.Nk, d, s, nu) * F_abs(f[d], f[s], N[p]) * gauss_delta(Dab, m->sigma_eph);
                }
            }
            dN[p] += -pref * acc;
        }
    }
    if ((parts & OR_PHPH) && m->pp_stride > 0) {
        or_pp pp;
        pp_init(m, &a, &pp);
        double pref = 36.0 * OR_PI / m->hbar / (double)pp.Nqs;
        double cut = 3.0 * m->sigma_pp;
#pragma omp parallel for schedule(dynamic, 4)
        for (long ia = 0; ia < pp.M; ++ia) {
            long pa = pp.full[ia];
            if (pmask && !pmask[pa]) continue;
            double wa = m->ph_omega[pa];
            if (wa < m->omega_cut) continue;
            int qa[3], qb[3];
            pp_coords(&pp, ia % pp.Nqs, qa);
            double acc = 0.0;
            for (long ib = 0; ib < pp.M; ++ib) {
                long pb = pp.full[ib];
                double wb = m->ph_omega[pb];
                if (wb < m->omega_cut) continue;
                pp_coords(&pp, ib % pp.Nqs, qb);
                long qem = pp_lin(&pp, wrap(qa[0] - qb[0], pp.nqs[0]), wrap(qa[1] - qb[1], pp.nqs[1]),
                                  wrap(qa[2] - qb[2], pp.nqs[2]));
                long qab = pp_lin(&pp, wrap(qb[0] - qa[0], pp.nqs[0]), wrap(qb[1] - qa[1], pp.nqs[1]),
                                  wrap(qb[2] - qa[2], pp.nqs[2]));
                for (int nu2 = 0; nu2 < m->nmodes; ++nu2) {
                    long pc = pp.full[(long)nu2 * pp.Nqs + qem];
                    double wc = m->ph_omega[pc];
                    if (wc >= m->omega_cut) {
                        double D = -wa + wb + wc;
                        if (fabs(D) <= cut)
                            acc += v3_of(m, &a, pa, pb, pc) * G_em(N[pa], N[pb], N[pc]) * gauss_delta(D, m->sigma_pp);
                    }
                    pc = pp.full[(long)nu2 * pp.Nqs + qab];
                    wc = m->ph_omega[pc];
                    if (wc >= m->omega_cut) {
                        double D = wa - wb + wc;
                        if (fabs(D) <= cut)
                            acc += 2.0 * v3_of(m, &a, pa, pb, pc) * G_abs(N[pa], N[pb], N[pc]) *
                                   gauss_delta(D, m->sigma_pp);
                    }
                }
            }
            dN[pa] += -pref * acc;
        }
        free(pp.full);
    }
    aux_free(&a);
}

/* ---------------------------------------------------------------------------
 * RHS from stored lists
 * ------------------------------------------------------------------------- */
typedef struct {
    const or_model *m;
    /* e-ph */
    const int64_t *eph_off; const int32_t *eph_src; const int32_t *eph_ph; const double *eph_W;
    /* ph-e (one segment per phonon, all N_ph phonons) */
    const int64_t *phe_off; const int32_t *phe_dst; const int32_t *phe_src; const double *phe_W;
    /* ph-ph */
    int64_t n_pp; const int64_t *pp_full; const int64_t *pp_off; const int32_t *pp_b; const int32_t *pp_c;
    const double *pp_W;
    unsigned parts;
    const double *forcing; /* optional vector added to ydot (MRI) */
    int64_t nrhs;
} or_problem;

void or_rhs_lists(const or_problem *P, const double *y, double *ydot, unsigned parts) {
    const or_model *m = P->m;
    long Nq = prod3(m->nq), Nph = (long)m->nmodes * Nq;
    const double *f = y, *N = y + m->n_c;
    double *df = ydot, *dN = ydot + m->n_c;
#pragma omp parallel for schedule(static)
    for (int d = 0; d < m->n_c; ++d) {
        double acc = 0.0;
        if (parts & OR_EPH) {
            for (long e = P->eph_off[2 * d]; e < P->eph_off[2 * d + 1]; ++e)
                acc += P->eph_W[e] * F_em(f[d], f[P->eph_src[e]], N[P->eph_ph[e]]);
            for (long e = P->eph_off[2 * d + 1]; e < P->eph_off[2 * d + 2]; ++e)
                acc += P->eph_W[e] * F_abs(f[d], f[P->eph_src[e]], N[P->eph_ph[e]]);
        }
        df[d] = -acc;
    }
#pragma omp parallel for schedule(static)
    for (long p = 0; p < Nph; ++p) {
        double acc = 0.0;
        if ((parts & OR_PHE) && P->phe_off)
            for (long e = P->phe_off[p]; e < P->phe_off[p + 1]; ++e)
                acc += P->phe_W[e] * F_abs(f[P->phe_dst[e]], f[P->phe_src[e]], N[p]);
        dN[p] = -acc;
    }
    if ((parts & OR_PHPH) && P->pp_off) {
#pragma omp parallel for schedule(dynamic, 16)
        for (long ia = 0; ia < P->n_pp; ++ia) {
            long pa = P->pp_full[ia];
            double acc = 0.0;
            for (long e = P->pp_off[2 * ia]; e < P->pp_off[2 * ia + 1]; ++e)
                acc += P->pp_W[e] * G_em(N[pa], N[P->pp_full[P->pp_b[e]]], N[P->pp_full[P->pp_c[e]]]);
            for (long e = P->pp_off[2 * ia + 1]; e < P->pp_off[2 * ia + 2]; ++e)
                acc += P->pp_W[e] * G_abs(N[pa], N[P->pp_full[P->pp_b[e]]], N[P->pp_full[P->pp_c[e]]]);
            dN[pa] += -acc;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Time integration (Methods B)
 * ------------------------------------------------------------------------- */
typedef void (*or_rhs_fn)(void *user, double t, const double *y, double *ydot);

/* Callback adapter: y' = RHS(parts) [+ forcing] for an or_problem. */
void or_problem_rhs(void *user, double t, const double *y, double *ydot) {
    or_problem *P = (or_problem *)user;
    (void)t;
    or_rhs_lists(P, y, ydot, P->parts);
    if (P->forcing) {
        long n = P->m->n_c + (long)P->m->nmodes * prod3(P->m->nq);
        for (long i = 0; i < n; ++i) ydot[i] += P->forcing[i];
    }
    P->nrhs++;
}

typedef struct {
    int S, p, has_emb;
    double A[6][6], b[6], bt[6], c[6];
} or_tableau;

enum { OR_RK4 = 0, OR_BS32 = 1, OR_ZON43 = 2, OR_KW3 = 3 };

static void tab_get(int id, or_tableau *T) {
    memset(T, 0, sizeof(*T));
    if (id == OR_RK4) { /* classical fourth-order Runge-Kutta */
        T->S = 4; T->p = 4; T->has_emb = 0;
        T->c[1] = 0.5; T->c[2] = 0.5; T->c[3] = 1.0;
        T->A[1][0] = 0.5; T->A[2][1] = 0.5; T->A[3][2] = 1.0;
        T->b[0] = 1.0 / 6; T->b[1] = 1.0 / 3; T->b[2] = 1.0 / 3; T->b[3] = 1.0 / 6;
    } else if (id == OR_BS32) { /* Bogacki-Shampine 3(2) */
        T->S = 4; T->p = 3; T->has_emb = 1;
        T->c[1] = 0.5; T->c[2] = 0.75; T->c[3] = 1.0;
        T->A[1][0] = 0.5;
        T->A[2][1] = 0.75;
        T->A[3][0] = 2.0 / 9; T->A[3][1] = 1.0 / 3; T->A[3][2] = 4.0 / 9;
        T->b[0] = 2.0 / 9; T->b[1] = 1.0 / 3; T->b[2] = 4.0 / 9; T->b[3] = 0.0;
        T->bt[0] = 7.0 / 24; T->bt[1] = 0.25; T->bt[2] = 1.0 / 3; T->bt[3] = 0.125;
    } else if (id == OR_ZON43) { /* Zonneveld 4(3), ARKODE's default explicit method */
        T->S = 5; T->p = 4; T->has_emb = 1;
        T->c[1] = 0.5; T->c[2] = 0.5; T->c[3] = 1.0; T->c[4] = 0.75;
        T->A[1][0] = 0.5;
        T->A[2][1] = 0.5;
        T->A[3][2] = 1.0;
        T->A[4][0] = 5.0 / 32; T->A[4][1] = 7.0 / 32; T->A[4][2] = 13.0 / 32; T->A[4][3] = -1.0 / 32;
        T->b[0] = 1.0 / 6; T->b[1] = 1.0 / 3; T->b[2] = 1.0 / 3; T->b[3] = 1.0 / 6; T->b[4] = 0.0;
        T->bt[0] = -0.5; T->bt[1] = 7.0 / 3; T->bt[2] = 7.0 / 3; T->bt[3] = 13.0 / 6; T->bt[4] = -16.0 / 3;
    } else if (id == OR_KW3) { /* Knoth-Wolke 3-stage, base of the MIS method */
        T->S = 3; T->p = 3; T->has_emb = 0;
        T->c[1] = 1.0 / 3; T->c[2] = 0.75;
        T->A[1][0] = 1.0 / 3;
        T->A[2][0] = -3.0 / 16; T->A[2][1] = 15.0 / 16;
        T->b[0] = 1.0 / 6; T->b[1] = 0.3; T->b[2] = 8.0 / 15;
    }
}

/* Exported so tests can check order conditions with exact rationals. */
void or_tableau_get(int id, int *S, int *p, double *A, double *b, double *bt, double *c) {
    or_tableau T;
    tab_get(id, &T);
    *S = T.S; *p = T.p;
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j < 6; ++j) A[i * 6 + j] = T.A[i][j];
        b[i] = T.b[i]; bt[i] = T.bt[i]; c[i] = T.c[i];
    }
}

typedef struct {
    int method;
    int pid_sign_mode;     /* 0: -a1,+a2,-a3 (ARKODE); 1: all negative (as printed) */
    double rtol;
    const double *atol;    /* [n] */
    double h0, hmin, hmax;
    int64_t max_steps;
    double a1, a2, a3;
    double safety, growth, growth_first, etamxf, etamin;
    int small_nef, max_nef;
} or_erk_opts;

typedef struct {
    int64_t steps, attempts, fails, rhs_evals, rhs_slow, slow_steps;
    double t, h_last, h_next;
    int status;
    int64_t slow_fails; /* rejected slow steps (tolerance-chosen slow step) */
} or_stats;

enum { OR_OK = 0, OR_TOO_MANY_STEPS = -4, OR_STEP_UNDERFLOW = -5, OR_ERR_TEST_FAIL = -6, OR_NONFINITE = -7 };

/* WRMS norm (Eq. wrms_norm) with weights from yref (Eq. wrms_weights). */
double or_wrms(long n, const double *v, const double *yref, double rtol, const double *atol) {
    double acc = 0.0;
    for (long i = 0; i < n; ++i) {
        double w = 1.0 / (rtol * fabs(yref[i]) + atol[i]);
        double x = v[i] * w;
        acc += x * x;
    }
    return sqrt(acc / (double)n);
}

/* Starting step (Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4), with the WRMS
 * norm of the integrator. Uses one extra RHS evaluation. */
static double h_start(or_rhs_fn fn, void *u, long n, double t0, const double *y0, const double *f0, double span,
                      int p, double rtol, const double *atol, double *tmp, double *tmp2, int64_t *nrhs) {
    double d0 = or_wrms(n, y0, y0, rtol, atol);
    double d1 = or_wrms(n, f0, y0, rtol, atol);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    if (h0 > span) h0 = span;
    for (long i = 0; i < n; ++i) tmp[i] = y0[i] + h0 * f0[i];
    fn(u, t0 + h0, tmp, tmp2);
    (*nrhs)++;
    for (long i = 0; i < n; ++i) tmp[i] = tmp2[i] - f0[i];
    double d2 = or_wrms(n, tmp, y0, rtol, atol) / h0;
    double dm = d1 > d2 ? d1 : d2;
    double h1 = dm <= 1e-15 ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 1.0 / (p + 1));
    double h = 100.0 * h0 < h1 ? 100.0 * h0 : h1;
    return h > span ? span : h;
}

/* Adaptive explicit RK (Eq. ERK_method) from t0 to t1 with PID control
 * (Eq. pid_controller).  y is overwritten with the solution at t1.
 * *h_io: in = initial step (<=0: estimate), out = next step proposal. */
int or_erk_solve(or_rhs_fn fn, void *u, long n, double t0, double t1, double *y, const or_erk_opts *o,
                 double *h_io, or_stats *st) {
    or_tableau T;
    tab_get(o->method, &T);
    int S = T.S, p = T.p;
    double *K = (double *)malloc(sizeof(double) * (size_t)n * (S + 4));
    double *z = K + (size_t)n * S, *ynew = z + n, *err = ynew + n, *tmp = err + n;
    double t = t0;
    double eps1 = 1.0, eps2 = 1.0;
    int first = 1, status = OR_OK;
    double h = h_io && *h_io > 0 ? *h_io : 0.0;
    if (h <= 0.0) {
        fn(u, t, y, K);
        st->rhs_evals++;
        h = h_start(fn, u, n, t, y, K, t1 - t0, p, o->rtol, o->atol, z, tmp, &st->rhs_evals);
    }
    if (o->hmax > 0 && h > o->hmax) h = o->hmax;
    int64_t steps = 0;
    int nef = 0;
    while (t < t1) {
        if (o->max_steps > 0 && steps >= o->max_steps) { status = OR_TOO_MANY_STEPS; break; }
        double hk = h;
        int last = 0;
        if (t + hk >= t1) { hk = t1 - t; last = 1; }
        for (int i = 0; i < S; ++i) {
            for (long r = 0; r < n; ++r) {
                double acc = 0.0;
                for (int j = 0; j < i; ++j) acc += T.A[i][j] * K[(size_t)j * n + r];
                z[r] = y[r] + hk * acc;
            }
            fn(u, t + T.c[i] * hk, z, K + (size_t)i * n);
            st->rhs_evals++;
        }
        int finite = 1;
        for (long r = 0; r < n; ++r) {
            double s1 = 0.0, s2 = 0.0;
            for (int i = 0; i < S; ++i) {
                s1 += T.b[i] * K[(size_t)i * n + r];
                s2 += (T.b[i] - T.bt[i]) * K[(size_t)i * n + r];
            }
            ynew[r] = y[r] + hk * s1;
            err[r] = hk * s2;
            if (!isfinite(ynew[r])) finite = 0;
        }
        st->attempts++;
        double eps = or_wrms(n, err, y, o->rtol, o->atol);
        if (!finite || !isfinite(eps)) { status = OR_NONFINITE; break; }
        if (eps <= 1.0) {
            memcpy(y, ynew, sizeof(double) * (size_t)n);
            t = last ? t1 : t + hk;
            steps++;
            st->steps++;
            double e = eps > 1e-10 ? eps : 1e-10;
            double e1 = eps1, e2 = eps2;
            double eta = o->pid_sign_mode == 0
                             ? pow(e, -o->a1 / p) * pow(e1, o->a2 / p) * pow(e2, -o->a3 / p)
                             : pow(e, -o->a1 / p) * pow(e1, -o->a2 / p) * pow(e2, -o->a3 / p);
            eta *= o->safety;
            double cap = first ? o->growth_first : o->growth;
            if (nef > 0 && cap > 1.0) cap = 1.0;
            if (eta > cap) eta = cap;
            h = hk * eta;
            if (o->hmax > 0 && h > o->hmax) h = o->hmax;
            eps2 = eps1;
            eps1 = e;
            first = 0;
            nef = 0;
            st->h_last = hk;
            if (t < t1 && !(t + h > t)) { status = OR_STEP_UNDERFLOW; break; }
        } else {
            st->fails++;
            nef++;
            if (nef >= o->max_nef) { status = OR_ERR_TEST_FAIL; break; }
            double eta = o->safety * pow(eps, -1.0 / p);
            if (eta < o->etamin) eta = o->etamin;
            if (eta > 1.0) eta = 1.0;
            if (nef >= o->small_nef && eta > o->etamxf) eta = o->etamxf;
            h = hk * eta;
            if (h < o->hmin || !(t + h > t)) { status = OR_STEP_UNDERFLOW; break; }
        }
    }
    st->t = t;
    st->h_next = h;
    st->status = status;
    if (h_io) *h_io = h;
    free(K);
    return status;
}

/* Fixed-step classical RK4 from t0 to t1 with step h (last step shortened). */
int or_rk4_solve(or_rhs_fn fn, void *u, long n, double t0, double t1, double h, double *y, or_stats *st) {
    or_tableau T;
    tab_get(OR_RK4, &T);
    double *K = (double *)malloc(sizeof(double) * (size_t)n * 5);
    double *z = K + (size_t)n * 4;
    double t = t0;
    long nsteps = (long)ceil((t1 - t0) / h - 1e-9);
    for (long k = 0; k < nsteps; ++k) {
        double hk = (k == nsteps - 1) ? t1 - t : h;
        for (int i = 0; i < 4; ++i) {
            for (long r = 0; r < n; ++r) {
                double acc = 0.0;
                for (int j = 0; j < i; ++j) acc += T.A[i][j] * K[(size_t)j * n + r];
                z[r] = y[r] + hk * acc;
            }
            fn(u, t + T.c[i] * hk, z, K + (size_t)i * n);
            st->rhs_evals++;
        }
        for (long r = 0; r < n; ++r) {
            double s = 0.0;
            for (int i = 0; i < 4; ++i) s += T.b[i] * K[(size_t)i * n + r];
            y[r] += hk * s;
        }
        t = (k == nsteps - 1) ? t1 : t + hk;
        st->steps++;
        st->attempts++;
    }
    st->t = t;
    free(K);
    for (long r = 0; r < n; ++r)
        if (!isfinite(y[r])) return st->status = OR_NONFINITE;
    return st->status = OR_OK;
}

/* MIS coupling coefficients (Eq. mis_coef, K = 1) for an S-stage base ERK method:
 * Om[i][j] for MRI stages i = 0..S (0-based), with the last row b_j - A_{S,j}. */
void or_mis_coef(int base, double *Om, double *chat) {
    or_tableau T;
    tab_get(base, &T);
    int S = T.S;
    memset(Om, 0, sizeof(double) * 6 * 6);
    for (int i = 0; i < S; ++i) chat[i] = T.c[i];
    chat[S] = 1.0;
    for (int i = 1; i < S; ++i)
        for (int j = 0; j < S; ++j) Om[i * 6 + j] = T.A[i][j] - T.A[i - 1][j];
    for (int j = 0; j < S; ++j) Om[S * 6 + j] = T.b[j] - T.A[S - 1][j];
}

typedef struct {
    or_rhs_fn ff;
    void *fu;
    const double *r;
    long n;
} or_forced;

static void forced_rhs(void *user, double t, const double *y, double *ydot) {
    or_forced *F = (or_forced *)user;
    F->ff(F->fu, t, y, ydot);
    for (long i = 0; i < F->n; ++i) ydot[i] += F->r[i];
}

/* One explicit MRI slow step (Methods B, algorithm steps 1-3) with MIS coupling on the
 * Knoth-Wolke base, from t over H: slow RHS at each stage start, constant forcing
 * r_i = (1/dc_i) sum_{j<i} Om_ij fs_j on the stage's sub-interval, fast auxiliary ODE solved by
 * the adaptive ERK of `inner`, which restarts its error history per stage and starts from the
 * carried proposal *h_in (0: estimate), clipped to the sub-interval.  Fs holds S + 1 vectors. */
static int mis_step(or_rhs_fn ff, void *fu, or_rhs_fn fs, void *su, long n, double t, double H, double *y,
                    const or_erk_opts *inner, double *h_in, double *Fs, or_stats *st) {
    double Om[36], chat[6];
    or_mis_coef(OR_KW3, Om, chat);
    const int S = 3;
    double *r = Fs + (size_t)n * S;
    or_forced F = {ff, fu, r, n};
    int status = OR_OK;
    fs(su, t, y, Fs); /* stage 1: z_1 = y */
    st->rhs_slow++;
    for (int i = 1; i <= S; ++i) {
        double dc = chat[i] - chat[i - 1];
        double ta = t + chat[i - 1] * H, tb = (i == S) ? t + H : t + chat[i] * H;
        for (long q = 0; q < n; ++q) {
            double acc = 0.0;
            for (int j = 0; j < i; ++j) acc += Om[i * 6 + j] * Fs[(size_t)j * n + q];
            r[q] = acc / dc;
        }
        if (*h_in > tb - ta) *h_in = tb - ta;
        or_stats in = {0};
        status = or_erk_solve(forced_rhs, &F, n, ta, tb, y, inner, h_in, &in);
        st->steps += in.steps;
        st->attempts += in.attempts;
        st->fails += in.fails;
        st->rhs_evals += in.rhs_evals;
        if (status != OR_OK) break;
        if (i < S) {
            fs(su, tb, y, Fs + (size_t)i * n);
            st->rhs_slow++;
        }
    }
    return status;
}

/* Explicit MRI with a fixed slow step hs (the last step ends at t1).  Each fast solve
 * restarts the error history; its first step is the previous fast solve's proposal
 * (estimated on the very first solve). */
int or_mri_solve(or_rhs_fn ff, void *fu, or_rhs_fn fs, void *su, long n, double t0, double t1, double hs, double *y,
                 const or_erk_opts *inner, or_stats *st) {
    double *Fs = (double *)malloc(sizeof(double) * (size_t)n * 4);
    double t = t0;
    double h_in = 0.0;
    int status = OR_OK;
    long nsteps = (long)ceil((t1 - t0) / hs - 1e-9);
    for (long k = 0; k < nsteps && status == OR_OK; ++k) {
        double H = (k == nsteps - 1) ? t1 - t : hs;
        status = mis_step(ff, fu, fs, su, n, t, H, y, inner, &h_in, Fs, st);
        t = (k == nsteps - 1) ? t1 : t + H;
        st->slow_steps++;
    }
    st->t = t;
    st->status = status;
    free(Fs);
    return status;
}

/* Slow-step control of the tolerance-chosen MRI (the method's stated extension: h_s chosen
 * from a tolerance instead of fixed).  Not in the paper; constants are library choices. */
typedef struct {
    double hs0;        /* first slow step                                              */
    double safety;     /* step factor safety (0.9)                                     */
    double fac_min;    /* smallest step factor (0.2)                                   */
    double fac_max;    /* largest step factor after an accepted step (5)               */
    double fast_scale; /* the fast ERK runs at rtol and atol times this (0.1)          */
    int max_fail;      /* consecutive rejected slow steps before giving up (7)         */
} or_slow_opts;

/* MRI (MIS on Knoth-Wolke, order 3) with the slow step chosen from the tolerance by step
 * doubling (Richardson extrapolation; Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4):
 * from the state y_n at t, one slow step of H gives y_1 and two of H/2 give y_2; the local
 * error of y_2 is estimated as (y_1 - y_2) / (2^3 - 1) and measured by the WRMS norm of
 * `inner`'s rtol / atol with weights from y_n (Eq. wrms_norm, Eq. wrms_weights).  eps <= 1
 * accepts y_2 and t + H; otherwise y_n is restored.  Next H = H * min(fac_max, max(fac_min,
 * safety * eps^(-1/4))), the factor capped at 1 after a rejection and on the attempt that
 * follows one.  The fast solves use rtol and atol scaled by fast_scale, so that their errors
 * stay below the slow estimate.  Both the single step and the first half step start from the
 * fast proposal held at y_n; an accepted step continues from the second half step's. */
int or_mri_adapt_solve(or_rhs_fn ff, void *fu, or_rhs_fn fs, void *su, long n, double t0, double t1,
                       const or_slow_opts *so, double *y, const or_erk_opts *inner, or_stats *st) {
    double *Fs = (double *)malloc(sizeof(double) * (size_t)n * 8);
    double *y0 = Fs + (size_t)n * 4, *y1 = y0 + n, *err = y1 + n, *atol_in = err + n;
    or_erk_opts in = *inner;
    in.rtol = inner->rtol * so->fast_scale;
    for (long i = 0; i < n; ++i) atol_in[i] = inner->atol[i] * so->fast_scale;
    in.atol = atol_in;
    double t = t0, H = so->hs0, h_in = 0.0;
    int status = OR_OK, nfail = 0, after_fail = 0;
    while (t < t1 && status == OR_OK) {
        if (inner->max_steps > 0 && st->slow_steps >= inner->max_steps) { status = OR_TOO_MANY_STEPS; break; }
        double Hk = H;
        int last = 0;
        if (t + Hk >= t1) { Hk = t1 - t; last = 1; }
        memcpy(y0, y, sizeof(double) * (size_t)n);
        const double h0 = h_in;
        /* one step of Hk */
        memcpy(y1, y0, sizeof(double) * (size_t)n);
        double hb = h0;
        status = mis_step(ff, fu, fs, su, n, t, Hk, y1, &in, &hb, Fs, st);
        if (status != OR_OK) break; /* y still holds y_n */
        /* two steps of Hk / 2 */
        const double Hh = 0.5 * Hk, tm = t + Hh;
        double hh = h0;
        status = mis_step(ff, fu, fs, su, n, t, Hh, y, &in, &hh, Fs, st);
        if (status == OR_OK) status = mis_step(ff, fu, fs, su, n, tm, Hh, y, &in, &hh, Fs, st);
        if (status != OR_OK) { /* hand back the last accepted state */
            memcpy(y, y0, sizeof(double) * (size_t)n);
            break;
        }
        int finite = 1;
        for (long i = 0; i < n; ++i) {
            err[i] = (y1[i] - y[i]) / 7.0; /* error of y_2: (y_1 - y_2) / (2^3 - 1) */
            if (!isfinite(y[i])) finite = 0;
        }
        double eps = or_wrms(n, err, y0, inner->rtol, inner->atol);
        if (!finite || !isfinite(eps)) { status = OR_NONFINITE; break; }
        if (eps <= 1.0) {
            t = last ? t1 : t + Hk;
            h_in = hh;
            st->slow_steps++;
            st->h_last = Hk;
            double e = eps > 1e-10 ? eps : 1e-10;
            double fac = so->safety * pow(e, -0.25);
            double cap = after_fail ? 1.0 : so->fac_max;
            if (fac > cap) fac = cap;
            if (fac < so->fac_min) fac = so->fac_min;
            H = Hk * fac;
            nfail = 0;
            after_fail = 0;
        } else {
            memcpy(y, y0, sizeof(double) * (size_t)n);
            h_in = h0;
            st->slow_fails++;
            if (++nfail >= so->max_fail) { status = OR_ERR_TEST_FAIL; break; }
            double fac = so->safety * pow(eps, -0.25);
            if (fac > 1.0) fac = 1.0;
            if (fac < so->fac_min) fac = so->fac_min;
            H = Hk * fac;
            after_fail = 1;
        }
        if (t < t1 && !(t + H > t)) { status = OR_STEP_UNDERFLOW; break; }
    }
    st->t = t;
    st->h_next = H;
    st->status = status;
    free(Fs);
    return status;
}

/* First-order operator splitting with RK4 (Results, Fig. 3 comparison): per step,
 * one RK4 step of the slow part with hs, then m = round(hs/hf) RK4 steps of the
 * fast part. */
int or_split_rk4_solve(or_rhs_fn ff, void *fu, or_rhs_fn fs, void *su, long n, double t0, double t1, double hs,
                       double hf, double *y, or_stats *st) {
    long nsteps = (long)ceil((t1 - t0) / hs - 1e-9);
    double t = t0;
    int status = OR_OK;
    for (long k = 0; k < nsteps && status == OR_OK; ++k) {
        double H = (k == nsteps - 1) ? t1 - t : hs;
        or_stats a = {0}, b = {0};
        status = or_rk4_solve(fs, su, n, t, t + H, H, y, &a);
        st->rhs_slow += a.rhs_evals;
        if (status != OR_OK) break;
        long m = (long)floor(H / hf + 0.5);
        if (m < 1) m = 1;
        status = or_rk4_solve(ff, fu, n, t, t + H, H / (double)m, y, &b);
        st->rhs_evals += b.rhs_evals;
        st->steps += 1;
        t = (k == nsteps - 1) ? t1 : t + H;
    }
    st->t = t;
    st->status = status;
    return status;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
