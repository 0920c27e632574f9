// builder.cu -- device construction of the stored scattering-channel lists.
//
// The paper stores the e-ph and ph-ph scattering "matrices" once, before the dynamics
// (Results, rt-BTE section), and sums them at every RHS evaluation.  This translation unit
// enumerates them on the GPU: one warp per destination scans every candidate source in
// index order, keeps a candidate when its energy mismatch is within 3 sigma and no phonon
// involved is below the frequency cutoff, and writes the kept entries in order using
// warp ballots (no sort pass).  The filter uses only IEEE FP64 subtraction/addition and
// comparisons on the host-supplied energy tables, and this file is compiled without FMA
// contraction, so the kept set and its enumeration order are bit-identical to any IEEE
// implementation of the same rule.  Two storage choices follow: the e-ph lists of a mode may
// be split into phonon-wavevector blocks (segments (mode, block, electron, process)) so that
// the populations a block reads fit in shared memory, and each full 128-entry block of a
// segment is then reordered for shared-memory banks (bank_order); downloads return every
// segment in enumeration order.
//
//   e-ph  (Eq. e-ph, first integral) destination d = (n, k), source s = (m, k'), mode nu,
//         q = T(k' - k).  Emission keeps |(eps_d - hw) - eps_s| <= 3 sigma; absorption
//         keeps |(eps_s - hw) - eps_d| <= 3 sigma (the second delta of Eq. e-ph, written with
//         the emitting state first so a pair's two entries see identical bits).
//         W = (2 pi / hbar)(1/N_q) |g|^2 delta(Delta).
//   ph-e  (Eq. e-ph, second integral) destination phonon p = (nu, q); entries are the
//         absorption processes d + p -> s with s at k_d + q; W = (4 pi / hbar)(1/N_k)|g|^2 delta.
//   ph-ph (Eq. ph-ph) destination a on the sub-lattice; emission a -> b + c with
//         q_c = q_a - q_b, stored once per unordered pair b <= c (weight doubled when
//         b != c since the ordered sum counts both); absorption a + c -> b with
//         q_c = q_b - q_a and weight 2 W; W = (36 pi / hbar)(1/N_q,pp) |V3|^2 delta.
//   delta(E) = exp(-(E/sigma)^2) / (sigma sqrt(pi)) (normalised Gaussian, Methods A).
#include <math.h>

#include <algorithm>
#include <cstring>

#include "internal.cuh"

namespace rtbte {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double gdelta(double E, double sigma) {
    double x = E / sigma;
    return exp(-x * x) / (sigma * sqrt(kPi));
}

__device__ __forceinline__ int q_index(const BuildTables &T, int4 kd, int4 ks) {
    int d0 = min_image(ks.x - kd.x, T.nk[0]);
    int d1 = min_image(ks.y - kd.y, T.nk[1]);
    int d2 = min_image(ks.z - kd.z, T.nk[2]);
    int q0 = wrapi(d0 / T.fold, T.nq[0]);
    int q1 = wrapi(d1 / T.fold, T.nq[1]);
    int q2 = wrapi(d2 / T.fold, T.nq[2]);
    return (q2 * T.nq[1] + q1) * T.nq[0] + q0;
}

__device__ __forceinline__ double w_eph(const BuildTables &T, int d, int s, int nu, double D, double pref) {
    unsigned long long u1 = T.eid[d], u2 = T.eid[s], v1 = T.eid_inv[d], v2 = T.eid_inv[s];
    unsigned long long lo = u1 < u2 ? u1 : u2, hi = u1 < u2 ? u2 : u1;
    unsigned long long ilo = v1 < v2 ? v1 : v2, ihi = v1 < v2 ? v2 : v1;
    if (ilo < lo || (ilo == lo && ihi < hi)) {
        lo = ilo;
        hi = ihi;
    }
    unsigned long long U = (unsigned long long)T.nbands * (unsigned long long)T.N_k;
    unsigned long long key = (lo * U + hi) * (unsigned long long)T.nmodes + (unsigned long long)nu;
    unsigned long long h = mix64(key ^ mix64(T.g2_seed));
    double g2 = T.g2[nu] * T.lut[h >> (64 - T.lut_bits)];
    return pref * g2 * gdelta(D, T.sigma_eph);
}

__device__ __forceinline__ void sort3u(unsigned long long &a, unsigned long long &b, unsigned long long &c) {
    unsigned long long x;
    if (a > b) { x = a; a = b; b = x; }
    if (b > c) { x = b; b = c; c = x; }
    if (a > b) { x = a; a = b; b = x; }
}

__device__ __forceinline__ double w_pp(const BuildTables &T, int a, int b, int c, double D) {
    unsigned long long t0 = T.pp_full[a], t1 = T.pp_full[b], t2 = T.pp_full[c];
    unsigned long long u0 = T.pp_full_inv[a], u1 = T.pp_full_inv[b], u2 = T.pp_full_inv[c];
    sort3u(t0, t1, t2);
    sort3u(u0, u1, u2);
    if (u0 < t0 || (u0 == t0 && (u1 < t1 || (u1 == t1 && u2 < t2)))) {
        t0 = u0;
        t1 = u1;
        t2 = u2;
    }
    unsigned long long N = (unsigned long long)T.N_ph;
    unsigned long long key = (t0 * N + t1) * N + t2;
    unsigned long long h = mix64(key ^ mix64(T.v3_seed));
    double v3 = T.v3 * T.lut[h >> (64 - T.lut_bits)];
    return T.pref_pp * v3 * gdelta(D, T.sigma_pp);
}

template <class R> __device__ __forceinline__ void put_w(void *W, long long i, double w) {
    reinterpret_cast<R *>(W)[i] = (R)w;
}

// Warp-inclusive prefix sum of small counts.
__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// ---- e-ph: one warp per destination d; segments (nu, d, proc) -----------------
template <bool FILL, class R>
__global__ void eph_enum(BuildTables T, long long *counts, const long long *off, uint32_t *idx, void *W) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (warp >= T.n_c) return;
    const int d = (int)warp;
    if (FILL && (d < T.row_lo || d >= T.row_hi)) return;  // row outside the slice: nothing stored
    const int4 kd = T.ek[d];
    const double ed = T.eps[d];
    const unsigned lt = (1u << lane) - 1u;
    // one scan of the sources per q-block: segments (mode, block, d, process), sources ascending
    for (int qb = 0; qb < T.eph_nqb; ++qb) {
    const int q_lo = qb * T.eph_qblk, q_hi = q_lo + T.eph_qblk;
    int run[2 * kMaxModes];
#pragma unroll
    for (int i = 0; i < 2 * kMaxModes; ++i) run[i] = 0;
    for (int base = 0; base < T.n_c; base += 32) {
        const int s = base + lane;
        int4 ks = s < T.n_c ? T.ek[s] : kd;
        double es = s < T.n_c ? T.eps[s] : 0.0;
        int q = q_index(T, kd, ks);
        const bool valid = s < T.n_c && q >= q_lo && q < q_hi;
#pragma unroll
        for (int nu = 0; nu < kMaxModes; ++nu) {
            if (nu >= T.nmodes) break;
            double w = T.omega[(long long)nu * T.N_q + q];
            bool live = valid && !(w < T.omega_cut);
            double Dem = __dsub_rn(__dsub_rn(ed, w), es);
            double Dab = __dsub_rn(__dsub_rn(es, w), ed);
            bool kem = live && Dem <= T.cut_eph && Dem >= -T.cut_eph;
            bool kab = live && Dab <= T.cut_eph && Dab >= -T.cut_eph;
            unsigned bem = __ballot_sync(kFull, kem), bab = __ballot_sync(kFull, kab);
            if (FILL) {
                long long seg = (((long long)nu * T.eph_nqb + qb) * T.n_c + d) * 2;
                if (kem) {
                    long long at = off[seg] + run[2 * nu] + __popc(bem & lt);
                    idx[at] = (uint32_t)s | ((uint32_t)q << T.s_bits);
                    put_w<R>(W, at, w_eph(T, d, s, nu, Dem, T.pref_eph));
                }
                if (kab) {
                    long long at = off[seg + 1] + run[2 * nu + 1] + __popc(bab & lt);
                    idx[at] = (uint32_t)s | ((uint32_t)q << T.s_bits);
                    put_w<R>(W, at, w_eph(T, d, s, nu, Dab, T.pref_eph));
                }
            }
            run[2 * nu] += __popc(bem);
            run[2 * nu + 1] += __popc(bab);
        }
    }
#pragma unroll
    for (int nu = 0; nu < kMaxModes; ++nu) {
        if (nu >= T.nmodes) break;
#pragma unroll
        for (int proc = 0; proc < 2; ++proc) {
            long long seg = (((long long)nu * T.eph_nqb + qb) * T.n_c + d) * 2 + proc;
            if (!FILL) {
                if (lane == 0) counts[seg] = run[2 * nu + proc];
            } else {  // zero-weight padding up to the next multiple of 4; its phonon index is the
                      // block's first q, so that its population read stays in the staged block
                long long a0 = off[seg] + run[2 * nu + proc], a1 = off[seg + 1];
                for (long long a = a0 + lane; a < a1; a += 32) {
                    idx[a] = (uint32_t)q_lo << T.s_bits;
                    put_w<R>(W, a, 0.0);
                }
            }
        }
    }
    }
}

// ---- ph-e: one warp per phonon p; entries (d, s) ordered by d then s --------------
constexpr int kMaxPre = 3;     // preimages per dimension of trunc(d/fold) = q (fold <= 2)
constexpr int kMaxCand = 96;   // kMaxPre^3 * nbands bound checked on the host

template <bool FILL, class R>
__global__ void phe_enum(BuildTables T, long long *counts, const long long *off, uint32_t *idx, void *W) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (warp >= T.N_ph) return;
    const long long p = warp;
    if (FILL && (T.n_c + p < T.row_lo || T.n_c + p >= T.row_hi)) return;  // row outside the slice
    const int nu = (int)(p / T.N_q);
    const int ql = (int)(p - (long long)nu * T.N_q);
    const double w = T.omega[p];
    int qc[3] = {ql % T.nq[0], (ql / T.nq[0]) % T.nq[1], ql / (T.nq[0] * T.nq[1])};
    // minimum-image displacements dd with trunc(dd / fold) = q_c (mod nq_c)
    int pre[3][kMaxPre], npre[3];
    for (int c = 0; c < 3; ++c) {
        npre[c] = 0;
        int n = T.nk[c];
        for (int dd = -(n - 1) / 2; dd <= n / 2; ++dd)
            if (wrapi(dd / T.fold, T.nq[c]) == qc[c] && npre[c] < kMaxPre) pre[c][npre[c]++] = dd;
    }
    long long run = 0;
    const bool live_p = !(w < T.omega_cut);
    for (int base = 0; base < T.n_c && live_p; base += 32) {
        const int d = base + lane;
        int cand[kMaxCand];
        int nc = 0;
        if (d < T.n_c) {
            int4 kd = T.ek[d];
            for (int b = 0; b < T.nbands; ++b)
                for (int i0 = 0; i0 < npre[0]; ++i0)
                    for (int i1 = 0; i1 < npre[1]; ++i1)
                        for (int i2 = 0; i2 < npre[2]; ++i2) {
                            int x = wrapi(kd.x + pre[0][i0], T.nk[0]);
                            int y = wrapi(kd.y + pre[1][i1], T.nk[1]);
                            int z = wrapi(kd.z + pre[2][i2], T.nk[2]);
                            long long kl = ((long long)z * T.nk[1] + y) * T.nk[0] + x;
                            int s = T.kmap[(long long)b * T.N_k + kl];
                            if (s >= 0 && nc < kMaxCand) cand[nc++] = s;
                        }
            // ascending source order (insertion sort of a handful of candidates)
            for (int i = 1; i < nc; ++i) {
                int v = cand[i], j = i - 1;
                while (j >= 0 && cand[j] > v) {
                    cand[j + 1] = cand[j];
                    --j;
                }
                cand[j + 1] = v;
            }
            // keep absorption-resonant ones
            int kept = 0;
            double ed = T.eps[d];
            for (int i = 0; i < nc; ++i) {
                double Dab = __dsub_rn(__dsub_rn(T.eps[cand[i]], w), ed);
                if (Dab <= T.cut_eph && Dab >= -T.cut_eph) cand[kept++] = cand[i];
            }
            nc = kept;
        }
        int incl = warp_incl_scan(nc, lane);
        int total = __shfl_sync(kFull, incl, 31);
        if (FILL && nc > 0) {
            long long at = off[p] + run + (incl - nc);
            double ed = T.eps[d];
            for (int i = 0; i < nc; ++i) {
                int s = cand[i];
                double Dab = __dsub_rn(__dsub_rn(T.eps[s], w), ed);
                idx[at + i] = (uint32_t)d | ((uint32_t)s << T.s_bits);
                put_w<R>(W, at + i, w_eph(T, d, s, nu, Dab, T.pref_phe));
            }
        }
        run += total;
    }
    if (!FILL) {
        if (lane == 0) counts[p] = run;
    } else {
        for (long long a = off[p] + run + lane; a < off[p + 1]; a += 32) {
            idx[a] = 0u;
            put_w<R>(W, a, 0.0);
        }
    }
}

// ---- ph-ph: one warp per sub-lattice destination a; segments (a, proc) ----------
template <bool FILL, class R>
__global__ void pp_enum(BuildTables T, long long *counts, const long long *off, uint32_t *idx, void *W) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (warp >= T.M) return;
    const int a = (int)warp;
    if (FILL && (T.n_c + T.pp_full[a] < T.row_lo || T.n_c + T.pp_full[a] >= T.row_hi)) return;  // outside the slice
    const double wa = T.omega[T.pp_full[a]];
    const int ql = (int)(a % T.N_qs);
    const int qa0 = ql % T.nqs[0], qa1 = (ql / T.nqs[0]) % T.nqs[1], qa2 = ql / (T.nqs[0] * T.nqs[1]);
    long long run[2] = {0, 0};
    const bool live_a = !(wa < T.omega_cut);
    for (int base = 0; base < T.M && live_a; base += 32) {
        const int b = base + lane;
        int cnt[2] = {0, 0};
        int cs[2][kMaxModes];
        double Dv[2][kMaxModes];
        double wb = 0.0;
        if (b < T.M) {
            wb = T.omega[T.pp_full[b]];
            if (!(wb < T.omega_cut)) {
                int qb = b % (int)T.N_qs;
                int qb0 = qb % T.nqs[0], qb1 = (qb / T.nqs[0]) % T.nqs[1], qb2 = qb / (T.nqs[0] * T.nqs[1]);
                for (int proc = 0; proc < 2; ++proc) {
                    int sg = proc == 0 ? 1 : -1;
                    int c0 = wrapi(sg * (qa0 - qb0), T.nqs[0]), c1 = wrapi(sg * (qa1 - qb1), T.nqs[1]),
                        c2 = wrapi(sg * (qa2 - qb2), T.nqs[2]);
                    int qcl = (c2 * T.nqs[1] + c1) * T.nqs[0] + c0;
                    for (int nu2 = 0; nu2 < T.nmodes; ++nu2) {
                        int c = nu2 * (int)T.N_qs + qcl;
                        if (proc == 0 && c < b) continue;
                        double wc = T.omega[T.pp_full[c]];
                        if (wc < T.omega_cut) continue;
                        double D = proc == 0 ? __dsub_rn(__dadd_rn(wb, wc), wa) : __dsub_rn(__dadd_rn(wa, wc), wb);
                        if (D <= T.cut_pp && D >= -T.cut_pp) {
                            cs[proc][cnt[proc]] = c;
                            Dv[proc][cnt[proc]] = D;
                            cnt[proc]++;
                        }
                    }
                }
            }
        }
        for (int proc = 0; proc < 2; ++proc) {
            int incl = warp_incl_scan(cnt[proc], lane);
            int total = __shfl_sync(kFull, incl, 31);
            if (FILL && cnt[proc] > 0) {
                long long at = off[2LL * a + proc] + run[proc] + (incl - cnt[proc]);
                for (int i = 0; i < cnt[proc]; ++i) {
                    int c = cs[proc][i];
                    double wv = w_pp(T, a, b, c, Dv[proc][i]);
                    wv = proc == 0 ? (b == c ? wv : 2.0 * wv) : 2.0 * wv;
                    idx[at + i] = (uint32_t)b | ((uint32_t)c << T.pp_bits);
                    put_w<R>(W, at + i, wv);
                }
            }
            run[proc] += total;
        }
    }
    for (int proc = 0; proc < 2; ++proc) {
        long long seg = 2LL * a + proc;
        if (!FILL) {
            if (lane == 0) counts[seg] = run[proc];
        } else {
            for (long long x = off[seg] + run[proc] + lane; x < off[seg + 1]; x += 32) {
                idx[x] = 0u;
                put_w<R>(W, x, 0.0);
            }
        }
    }
}

template <class T> int dev_upload(rtbte_ctx *ctx, DevBuf &b, const std::vector<T> &h) {
    b.release();
    size_t bytes = std::max<size_t>(h.size() * sizeof(T), 16);
    RT_CUDA(ctx, cudaMalloc(&b.p, bytes));
    b.bytes = bytes;
    if (!h.empty()) RT_CUDA(ctx, cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return RTBTE_OK;
}

// Bank-aware entry order.  The collision kernel gives lane l of a warp the 16-byte vector l of
// each 128-entry block of an item and gathers, for component k of every vector, two populations
// from shared memory per entry; 32 lanes whose gather addresses share a bank serialise.  Each
// full block of a segment that lies inside its logical entries (blocks counted from the segment
// start, as the work items are) is reordered so that position 4*l + k holds the entry a greedy
// assigns to lane l and component k: entries in built order, each to the component whose lanes
// so far use neither of its two banks (else the one with fewer clashes, then the lowest).  The
// block holding the segment's last logical entry and its padding keeps the built order, so
// padding stays at the segment end.  Sums over a segment do not depend on its entry order
// beyond rounding; rtbte_download_channels returns every segment in its sorted order.
template <class R>
__global__ void bank_order(uint32_t *idx, R *W, const long long *off, const long long *cnt, long long nseg, int part,
                           int lo_bits, int nc, int nqb, int qblk, int l0) {
    const long long seg = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (seg >= nseg) return;
    constexpr int NB = sizeof(R) == 4 ? 32 : 16;  // banks per shared-memory element size
    const long long b0 = off[seg], n = cnt[seg];
    const unsigned lmask = (1u << lo_bits) - 1u;
    int offB = 0;  // element offset of the second gather's array in shared memory
    if (part == PART_EPH) {
        const long long blk = seg / (2LL * nc);
        offB = l0 - (int)(blk % nqb) * qblk;
    }
    uint32_t ib[128];
    R wb[128];
    for (long long c0 = 0; c0 + 128 <= n; c0 += 128) {
        for (int i = 0; i < 128; ++i) {
            ib[i] = idx[b0 + c0 + i];
            wb[i] = W[b0 + c0 + i];
        }
        unsigned mA[4] = {0u, 0u, 0u, 0u}, mB[4] = {0u, 0u, 0u, 0u};
        int fill[4] = {0, 0, 0, 0};
        for (int i = 0; i < 128; ++i) {
            const uint32_t e = ib[i];
            const int ba = (int)((e & lmask) % NB);
            const int bb = (int)((((long long)(e >> lo_bits) + offB) % NB + NB) % NB);
            int best = -1, cost = 3;
            for (int k = 0; k < 4; ++k) {
                if (fill[k] >= 32) continue;
                const int c = (int)((mA[k] >> ba) & 1u) + (int)((mB[k] >> bb) & 1u);
                if (c < cost) {
                    cost = c;
                    best = k;
                }
            }
            const int lane = fill[best]++;
            mA[best] |= 1u << ba;
            mB[best] |= 1u << bb;
            if (fill[best] == 32) mA[best] = mB[best] = ~0u;  // full: never chosen again
            const long long at = b0 + c0 + 4 * lane + best;
            idx[at] = e;
            W[at] = wb[i];
        }
    }
}

template <class R>
int order_banks(rtbte_ctx *ctx, const InstHost &I, int part, DevBuf &idx, DevBuf &W, const DevBuf &off,
                const DevBuf &cnt, long long nseg) {
    if (nseg <= 0) return RTBTE_OK;
    const int lo_bits = part == PART_PP ? I.pp_bits : I.s_bits;
    bank_order<R><<<(unsigned)((nseg + 127) / 128), 128, 0, ctx->stream>>>(
        idx.as<uint32_t>(), W.as<R>(), off.as<long long>(), cnt.as<long long>(), nseg, part, lo_bits, I.d.n_c,
        std::max(I.eph_nqb, 1), I.eph_qblk > 0 ? I.eph_qblk : I.N_q_pad, I.n_c_pad);
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    return RTBTE_OK;
}

// counts -> padded offsets; returns total stored entries
long long pad_offsets(const std::vector<long long> &cnt, std::vector<long long> &off) {
    off.assign(cnt.size() + 1, 0);
    for (size_t i = 0; i < cnt.size(); ++i) off[i + 1] = off[i] + round_up(cnt[i], kSegPad);
    return off.back();
}

BuildTables tables_of(rtbte_ctx *ctx, InstHost &I) {
    BuildTables T{};
    T.ek = I.t_ek.as<int4>();
    T.eps = I.t_eps.as<double>();
    T.eid = I.t_eid.as<unsigned long long>();
    T.eid_inv = I.t_eidinv.as<unsigned long long>();
    T.omega = I.t_omega.as<double>();
    T.kmap = I.t_kmap.as<int>();
    T.lut = I.t_lut.as<double>();
    T.g2 = I.t_g2.as<double>();
    T.pp_full = I.t_ppfull.as<int>();
    T.pp_full_inv = I.t_ppinv.as<int>();
    T.n_c = I.d.n_c;
    T.nbands = I.d.nbands;
    T.nmodes = I.d.nmodes;
    T.fold = I.d.fold;
    T.lut_bits = I.d.lut_bits;
    for (int c = 0; c < 3; ++c) {
        T.nk[c] = I.d.nk[c];
        T.nq[c] = I.d.nq[c];
        T.nqs[c] = I.nqs[c];
    }
    T.N_k = I.N_k;
    T.N_q = I.N_q;
    T.N_ph = I.n_ph;
    T.M = I.M;
    T.N_qs = I.N_qs;
    T.s_bits = I.s_bits;
    T.q_bits = I.q_bits;
    T.pp_bits = I.pp_bits;
    T.eph_nqb = I.eph_nqb;
    T.eph_qblk = I.eph_qblk;
    T.row_lo = I.row_lo;
    T.row_hi = I.row_hi;
    T.sigma_eph = I.d.sigma_eph;
    T.sigma_pp = I.d.sigma_pp;
    T.cut_eph = 3.0 * I.d.sigma_eph;
    T.cut_pp = 3.0 * I.d.sigma_pp;
    T.omega_cut = I.d.omega_cut;
    T.pref_eph = 2.0 * kPi / ctx->hbar / (double)I.N_q;
    T.pref_phe = 4.0 * kPi / ctx->hbar / (double)I.N_k;
    T.pref_pp = I.M > 0 ? 36.0 * kPi / ctx->hbar / (double)I.N_qs : 0.0;
    T.v3 = I.d.v3_coef;
    T.g2_seed = I.d.g2_seed;
    T.v3_seed = I.d.v3_seed;
    return T;
}

// e-ph q-blocks of instance I: one when f and one mode's N fit in shared memory together (or
// when f alone leaves under 16 KB, and the kernel reads populations from global memory anyway),
// else the fewest equal blocks of whole multiples of 4 q points that fit; a count requested at
// creation overrides the choice.
void choose_q_blocks(rtbte_ctx *ctx, InstHost &I) {
    const long long R = (long long)ctx->real_size;
    const long long room = (long long)ctx->smem_optin - 64 - (long long)I.n_c_pad * R;
    long long nqb = 1;
    if (ctx->eph_q_blocks > 0)
        nqb = ctx->eph_q_blocks;
    else if ((long long)I.N_q_pad * R > room && room >= 16384)
        nqb = ((long long)I.N_q_pad * R + room - 1) / room;
    long long qblk = round_up((I.N_q + nqb - 1) / nqb, 4);
    nqb = (I.N_q + qblk - 1) / qblk;
    I.eph_nqb = (int)std::max<long long>(nqb, 1);
    I.eph_qblk = (int)std::max<long long>(qblk, 4);
}

// Counts of every segment (all rows) -> padded lengths kept for the plan's lane choice; counts
// of segments whose destination row lies outside the instance's row slice are then zeroed
// (also on the device, where the bank-order pass reads them).  row_of(g) = state row of g.
template <class RowOf>
int slice_counts(rtbte_ctx *ctx, const InstHost &I, std::vector<long long> &cnt, std::vector<long long> &plen,
                 DevBuf &dcnt, RowOf row_of) {
    plen.resize(cnt.size());
    bool cut = false;
    for (size_t g = 0; g < cnt.size(); ++g) {
        plen[g] = round_up(cnt[g], kSegPad);
        const long long r = row_of((long long)g);
        if (r < I.row_lo || r >= I.row_hi) {
            cut = cut || cnt[g] != 0;
            cnt[g] = 0;
        }
    }
    if (cut && !cnt.empty())
        RT_CUDA(ctx, cudaMemcpyAsync(dcnt.p, cnt.data(), sizeof(long long) * cnt.size(), cudaMemcpyHostToDevice,
                                     ctx->stream));
    return RTBTE_OK;
}

template <class R>
int run_build(rtbte_ctx *ctx, InstHost &I, bool count_only) {
    BuildTables T = tables_of(ctx, I);
    const int threads = 256, wpb = threads / 32;
    DevBuf cnt, off;
    // ---- e-ph, in q-blocks when f and a whole mode's N do not fit in shared memory together
    choose_q_blocks(ctx, I);
    T.eph_nqb = I.eph_nqb;
    T.eph_qblk = I.eph_qblk;
    long long nseg = 2LL * I.d.nmodes * I.eph_nqb * I.d.n_c;
    RT_CUDA(ctx, cudaMalloc(&cnt.p, sizeof(long long) * std::max<long long>(nseg, 1)));
    eph_enum<false, R><<<(unsigned)((I.d.n_c + wpb - 1) / wpb), threads, 0, ctx->stream>>>(T, cnt.as<long long>(),
                                                                                          nullptr, nullptr, nullptr);
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    I.eph_cnt.assign(nseg, 0);
    RT_CUDA(ctx, cudaMemcpyAsync(I.eph_cnt.data(), cnt.p, sizeof(long long) * nseg, cudaMemcpyDeviceToHost, ctx->stream));
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int rc;
    const long long nc = I.d.n_c;
    if (count_only) {
        cnt.release();
        I.eph_off.clear();
    } else {
        if ((rc = slice_counts(ctx, I, I.eph_cnt, I.eph_plen, cnt, [&](long long g) { return (g / 2) % nc; })))
            return rc;
    }
    long long E = count_only ? 0 : pad_offsets(I.eph_cnt, I.eph_off);
    if (!count_only) {
    I.eph_idx.release();
    I.eph_W.release();
    RT_CUDA(ctx, cudaMalloc(&I.eph_idx.p, sizeof(uint32_t) * std::max<long long>(E, 4)));
    RT_CUDA(ctx, cudaMalloc(&I.eph_W.p, sizeof(R) * std::max<long long>(E, 4)));
    I.eph_idx.bytes = sizeof(uint32_t) * std::max<long long>(E, 4);
    I.eph_W.bytes = sizeof(R) * std::max<long long>(E, 4);
    if (dev_upload(ctx, off, I.eph_off)) return RTBTE_E_CUDA;
    eph_enum<true, R><<<(unsigned)((I.d.n_c + wpb - 1) / wpb), threads, 0, ctx->stream>>>(
        T, nullptr, off.as<long long>(), I.eph_idx.as<uint32_t>(), I.eph_W.p);
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    if ((rc = order_banks<R>(ctx, I, PART_EPH, I.eph_idx, I.eph_W, off, cnt, nseg))) return rc;
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cnt.release();
    off.release();
    }
    // ---- ph-e
    long long nph = I.n_ph;
    RT_CUDA(ctx, cudaMalloc(&cnt.p, sizeof(long long) * std::max<long long>(nph, 1)));
    phe_enum<false, R><<<(unsigned)((nph + wpb - 1) / wpb), threads, 0, ctx->stream>>>(T, cnt.as<long long>(), nullptr,
                                                                                     nullptr, nullptr);
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    I.phe_cnt.assign(nph, 0);
    RT_CUDA(ctx, cudaMemcpyAsync(I.phe_cnt.data(), cnt.p, sizeof(long long) * nph, cudaMemcpyDeviceToHost, ctx->stream));
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (count_only) {
        cnt.release();
        I.phe_off.clear();
    } else {
    if ((rc = slice_counts(ctx, I, I.phe_cnt, I.phe_plen, cnt, [&](long long g) { return nc + g; }))) return rc;
    E = pad_offsets(I.phe_cnt, I.phe_off);
    I.phe_idx.release();
    I.phe_W.release();
    RT_CUDA(ctx, cudaMalloc(&I.phe_idx.p, sizeof(uint32_t) * std::max<long long>(E, 4)));
    RT_CUDA(ctx, cudaMalloc(&I.phe_W.p, sizeof(R) * std::max<long long>(E, 4)));
    I.phe_idx.bytes = sizeof(uint32_t) * std::max<long long>(E, 4);
    I.phe_W.bytes = sizeof(R) * std::max<long long>(E, 4);
    if (dev_upload(ctx, off, I.phe_off)) return RTBTE_E_CUDA;
    phe_enum<true, R><<<(unsigned)((nph + wpb - 1) / wpb), threads, 0, ctx->stream>>>(
        T, nullptr, off.as<long long>(), I.phe_idx.as<uint32_t>(), I.phe_W.p);
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    if ((rc = order_banks<R>(ctx, I, PART_PHE, I.phe_idx, I.phe_W, off, cnt, nph))) return rc;
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cnt.release();
    off.release();
    }
    // ---- ph-ph
    I.pp_cnt.clear();
    I.pp_off.assign(1, 0);
    I.pp_off_dev.release();
    I.pp_idx.release();
    I.pp_W.release();
    if (I.M > 0) {
        long long ns = 2 * I.M;
        RT_CUDA(ctx, cudaMalloc(&cnt.p, sizeof(long long) * ns));
        pp_enum<false, R><<<(unsigned)((I.M + wpb - 1) / wpb), threads, 0, ctx->stream>>>(T, cnt.as<long long>(),
                                                                                        nullptr, nullptr, nullptr);
        RT_CUDA(ctx, cudaGetLastError());
        ctx->launches++;
        I.pp_cnt.assign(ns, 0);
        RT_CUDA(ctx, cudaMemcpyAsync(I.pp_cnt.data(), cnt.p, sizeof(long long) * ns, cudaMemcpyDeviceToHost, ctx->stream));
        RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (count_only) {
            cnt.release();
            I.pp_off.assign(1, 0);
            return RTBTE_OK;
        }
        if ((rc = slice_counts(ctx, I, I.pp_cnt, I.pp_plen, cnt,
                               [&](long long g) { return nc + (long long)I.pp_full[g / 2]; })))
            return rc;
        E = pad_offsets(I.pp_cnt, I.pp_off);
        RT_CUDA(ctx, cudaMalloc(&I.pp_idx.p, sizeof(uint32_t) * std::max<long long>(E, 4)));
        RT_CUDA(ctx, cudaMalloc(&I.pp_W.p, sizeof(R) * std::max<long long>(E, 4)));
        I.pp_idx.bytes = sizeof(uint32_t) * std::max<long long>(E, 4);
        I.pp_W.bytes = sizeof(R) * std::max<long long>(E, 4);
        if (dev_upload(ctx, off, I.pp_off)) return RTBTE_E_CUDA;
        pp_enum<true, R><<<(unsigned)((I.M + wpb - 1) / wpb), threads, 0, ctx->stream>>>(
            T, nullptr, off.as<long long>(), I.pp_idx.as<uint32_t>(), I.pp_W.p);
        RT_CUDA(ctx, cudaGetLastError());
        ctx->launches++;
        if ((rc = order_banks<R>(ctx, I, PART_PP, I.pp_idx, I.pp_W, off, cnt, ns))) return rc;
        RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cnt.release();
        off.release();
    }
    return RTBTE_OK;
}

}  // namespace

// Copy the instance's model tables to the device (builder inputs).
int upload_tables(rtbte_ctx *ctx, int i) {
    InstHost &I = ctx->inst[i];
    const int nc = I.d.n_c;
    std::vector<int4> ek(nc);
    std::vector<unsigned long long> eid(nc), einv(nc);
    for (int s = 0; s < nc; ++s) {
        int x = I.e_k[3 * s], y = I.e_k[3 * s + 1], z = I.e_k[3 * s + 2], b = I.e_band[s];
        ek[s] = make_int4(x, y, z, b);
        long long kl = ((long long)z * I.d.nk[1] + y) * I.d.nk[0] + x;
        long long ki = ((long long)wrapi(-z, I.d.nk[2]) * I.d.nk[1] + wrapi(-y, I.d.nk[1])) * I.d.nk[0] +
                       wrapi(-x, I.d.nk[0]);
        eid[s] = (unsigned long long)b * (unsigned long long)I.N_k + (unsigned long long)kl;
        einv[s] = (unsigned long long)b * (unsigned long long)I.N_k + (unsigned long long)ki;
    }
    std::vector<int> kmap((size_t)I.d.nbands * I.N_k, -1);
    for (int s = 0; s < nc; ++s) kmap[(size_t)I.e_band[s] * I.N_k + (eid[s] - (unsigned long long)I.e_band[s] * I.N_k)] = s;
    int rc;
    if ((rc = dev_upload(ctx, I.t_ek, ek))) return rc;
    if ((rc = dev_upload(ctx, I.t_eps, I.e_eps))) return rc;
    if ((rc = dev_upload(ctx, I.t_eid, eid))) return rc;
    if ((rc = dev_upload(ctx, I.t_eidinv, einv))) return rc;
    if ((rc = dev_upload(ctx, I.t_omega, I.ph_omega))) return rc;
    if ((rc = dev_upload(ctx, I.t_kmap, kmap))) return rc;
    if ((rc = dev_upload(ctx, I.t_lut, I.lut))) return rc;
    if ((rc = dev_upload(ctx, I.t_g2, I.g2_coef))) return rc;
    if ((rc = dev_upload(ctx, I.t_ppfull, I.pp_full))) return rc;
    if ((rc = dev_upload(ctx, I.t_ppinv, I.pp_full_inv))) return rc;
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RTBTE_OK;
}

int build_channels(rtbte_ctx *ctx, int i, bool count_only) {
    InstHost &I = ctx->inst[i];
    if (I.d.nbands * kMaxPre * kMaxPre * kMaxPre > kMaxCand && I.d.fold > 1)
        return fail(ctx, RTBTE_E_UNSUPPORTED, "too many bands for the folded ph-e candidate buffer");
    if (I.d.nbands > kMaxCand) return fail(ctx, RTBTE_E_UNSUPPORTED, "too many bands");
    if (count_only) {  // nothing stored: the lists of an earlier upload go
        DevBuf *bufs[] = {&I.eph_idx, &I.eph_W, &I.phe_idx, &I.phe_W, &I.pp_idx, &I.pp_W, &I.pp_off_dev};
        for (DevBuf *b : bufs) b->release();
    }
    int rc = ctx->precision == RTBTE_PREC_FP64 ? run_build<double>(ctx, I, count_only)
                                               : run_build<float>(ctx, I, count_only);
    if (rc) return rc;
    I.counted = true;
    I.has_channels = !count_only;
    return RTBTE_OK;
}

}  // namespace rtbte
