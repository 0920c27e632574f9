// api.cu -- the extern "C" boundary of librtbte (declared in include/rtbte.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

namespace rtbte {

// NVTX range over a public call (visible to profilers; no cost without a tool attached)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

int fail(rtbte_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(rtbte_ctx *ctx, cudaError_t e, const char *what) {
    if (ctx) ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // clear a non-sticky error so the context stays usable
    return RTBTE_E_CUDA;
}

namespace {

int dev_alloc(rtbte_ctx *ctx, DevBuf &b, size_t bytes, bool zero) {
    b.release();
    bytes = std::max<size_t>(bytes, 16);
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ctx, RTBTE_E_OOM, "device allocation failed");
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    b.bytes = bytes;
    if (zero) RT_CUDA(ctx, cudaMemsetAsync(b.p, 0, bytes, ctx->stream));
    return RTBTE_OK;
}

bool ptr_is_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int setup_instance(rtbte_ctx *ctx, const rtbte_instance_desc &d, InstHost &I) {
    if (d.dim < 2 || d.dim > 3 || d.nbands < 1 || d.nmodes < 1 || d.nmodes > kMaxModes || d.n_c < 1 ||
        d.fold < 1 || d.fold > 2 || d.lut_bits < 1 || d.lut_bits > 20)
        return fail(ctx, RTBTE_E_INVALID_ARG, "instance descriptor out of range");
    if (!d.e_band || !d.e_k || !d.e_eps || !d.ph_omega || !d.lut || !d.g2_coef)
        return fail(ctx, RTBTE_E_INVALID_ARG, "instance descriptor has a NULL table");
    if (!(d.sigma_eph > 0) || (d.pp_stride > 0 && !(d.sigma_pp > 0)) || !(d.omega_cut >= 0))
        return fail(ctx, RTBTE_E_INVALID_ARG, "broadening and cutoff must be positive");
    for (int c = 0; c < 3; ++c) {
        if (d.nk[c] < 1 || d.nq[c] < 1) return fail(ctx, RTBTE_E_INVALID_ARG, "grid sizes must be >= 1");
        if (d.nk[c] > 1 && d.nk[c] != d.nq[c] * d.fold) return fail(ctx, RTBTE_E_INVALID_ARG, "nk must equal fold*nq");
        if (d.nk[c] == 1 && d.nq[c] != 1) return fail(ctx, RTBTE_E_INVALID_ARG, "flat dimension mismatch");
    }
    I.d = d;
    I.N_k = (long long)d.nk[0] * d.nk[1] * d.nk[2];
    I.N_q = (long long)d.nq[0] * d.nq[1] * d.nq[2];
    I.n_ph = (long long)d.nmodes * I.N_q;
    I.e_band.assign(d.e_band, d.e_band + d.n_c);
    I.e_k.assign(d.e_k, d.e_k + 3LL * d.n_c);
    I.e_eps.assign(d.e_eps, d.e_eps + d.n_c);
    I.ph_omega.assign(d.ph_omega, d.ph_omega + I.n_ph);
    I.lut.assign(d.lut, d.lut + (1LL << d.lut_bits));
    I.g2_coef.assign(d.g2_coef, d.g2_coef + d.nmodes);
    for (int s = 0; s < d.n_c; ++s) {
        if (I.e_band[s] < 0 || I.e_band[s] >= d.nbands) return fail(ctx, RTBTE_E_INVALID_ARG, "band index out of range");
        for (int c = 0; c < 3; ++c)
            if (I.e_k[3 * s + c] < 0 || I.e_k[3 * s + c] >= d.nk[c])
                return fail(ctx, RTBTE_E_INVALID_ARG, "k coordinate out of range");
    }
    I.s_bits = bits_for(d.n_c);
    I.q_bits = bits_for(I.N_q);
    if (I.s_bits + I.q_bits > 32 || 2 * I.s_bits > 32)
        return fail(ctx, RTBTE_E_UNSUPPORTED, "electron/phonon counts exceed the 32-bit e-ph entry format");
    I.N_q_pad = (int)round_up(I.N_q, 4);
    I.n_c_pad = (int)round_up(d.n_c, 4);
    I.compact.assign(I.n_ph, -1);
    I.pp_full.clear();
    I.pp_full_inv.clear();
    I.M = 0;
    I.N_qs = 0;
    if (d.pp_stride > 0) {
        const int st = d.pp_stride;
        for (int c = 0; c < 3; ++c) {
            if (d.nq[c] > 1 && d.nq[c] % st != 0) return fail(ctx, RTBTE_E_INVALID_ARG, "pp_stride must divide nq");
            I.nqs[c] = d.nq[c] > 1 ? d.nq[c] / st : 1;
        }
        I.N_qs = (long long)I.nqs[0] * I.nqs[1] * I.nqs[2];
        I.M = (long long)d.nmodes * I.N_qs;
        I.pp_bits = bits_for(I.M);
        if (2 * I.pp_bits > 32) return fail(ctx, RTBTE_E_UNSUPPORTED, "sub-lattice too large for the ph-ph entry format");
        I.pp_full.resize(I.M);
        I.pp_full_inv.resize(I.M);
        for (int nu = 0; nu < d.nmodes; ++nu)
            for (long long ql = 0; ql < I.N_qs; ++ql) {
                int x = (int)(ql % I.nqs[0]), y = (int)((ql / I.nqs[0]) % I.nqs[1]),
                    z = (int)(ql / ((long long)I.nqs[0] * I.nqs[1]));
                int sx = d.nq[0] > 1 ? st : 1, sy = d.nq[1] > 1 ? st : 1, sz = d.nq[2] > 1 ? st : 1;
                int X = x * sx, Y = y * sy, Z = z * sz;
                long long a = (long long)nu * I.N_qs + ql;
                long long full = (long long)nu * I.N_q + ((long long)Z * d.nq[1] + Y) * d.nq[0] + X;
                long long finv = (long long)nu * I.N_q +
                                 ((long long)wrapi(-Z, d.nq[2]) * d.nq[1] + wrapi(-Y, d.nq[1])) * d.nq[0] +
                                 wrapi(-X, d.nq[0]);
                I.pp_full[a] = (int32_t)full;
                I.pp_full_inv[a] = (int32_t)finv;
                I.compact[full] = (int32_t)a;
            }
    }
    I.M_pad = (int)round_up(I.M, 4);
    return RTBTE_OK;
}

template <class R>
int upload_prebuilt(rtbte_ctx *ctx, InstHost &I, const rtbte_channels *ch) {
    const int nc = I.d.n_c, nm = I.d.nmodes;
    // row_of(g): state row of segment g; segments outside the row slice are stored empty
    auto pack = [&](long long nseg, const int64_t *off, auto encode, auto row_of, std::vector<long long> &cnt,
                    std::vector<long long> &plen, std::vector<long long> &poff, DevBuf &didx, DevBuf &dW,
                    const double *W) -> int {
        cnt.assign(nseg, 0);
        plen.assign(nseg, 0);
        poff.assign(nseg + 1, 0);
        for (long long g = 0; g < nseg; ++g) {
            long long c = off[g + 1] - off[g];
            if (c < 0) return fail(ctx, RTBTE_E_INVALID_ARG, "offsets must be non-decreasing");
            plen[g] = round_up(c, kSegPad);
            const long long r = row_of(g);
            cnt[g] = (r >= I.row_lo && r < I.row_hi) ? c : 0;
            poff[g + 1] = poff[g] + round_up(cnt[g], kSegPad);
        }
        const long long E = poff[nseg];
        std::vector<uint32_t> hidx(std::max<long long>(E, 4), 0u);
        std::vector<R> hW(std::max<long long>(E, 4), R(0));
        for (long long g = 0; g < nseg; ++g)
            for (long long k = 0; k < cnt[g]; ++k) {
                uint32_t code;
                if (!encode(g, off[g] + k, &code)) return fail(ctx, RTBTE_E_INVALID_ARG, "channel index out of range");
                hidx[poff[g] + k] = code;
                hW[poff[g] + k] = (R)W[off[g] + k];
            }
        didx.release();
        dW.release();
        RT_CUDA(ctx, cudaMalloc(&didx.p, hidx.size() * sizeof(uint32_t)));
        RT_CUDA(ctx, cudaMalloc(&dW.p, hW.size() * sizeof(R)));
        didx.bytes = hidx.size() * sizeof(uint32_t);
        dW.bytes = hW.size() * sizeof(R);
        RT_CUDA(ctx, cudaMemcpy(didx.p, hidx.data(), didx.bytes, cudaMemcpyHostToDevice));
        RT_CUDA(ctx, cudaMemcpy(dW.p, hW.data(), dW.bytes, cudaMemcpyHostToDevice));
        return RTBTE_OK;
    };
    if (!ch->eph_off || !ch->phe_off) return fail(ctx, RTBTE_E_INVALID_ARG, "prebuilt e-ph and ph-e lists required");
    I.eph_nqb = 1;  // prebuilt e-ph lists: segments (mode, electron, process)
    I.eph_qblk = I.N_q_pad;
    int rc;
    rc = pack(2LL * nm * nc, ch->eph_off,
              [&](long long g, long long e, uint32_t *code) {
                  const int nu = (int)(g / (2LL * nc));
                  const int s = ch->eph_src[e];
                  const long long q = (long long)ch->eph_ph[e] - (long long)nu * I.N_q;
                  if (s < 0 || s >= nc || q < 0 || q >= I.N_q) return false;
                  *code = (uint32_t)s | ((uint32_t)q << I.s_bits);
                  return true;
              },
              [&](long long g) { return (g / 2) % nc; }, I.eph_cnt, I.eph_plen, I.eph_off, I.eph_idx, I.eph_W,
              ch->eph_W);
    if (rc) return rc;
    rc = pack(I.n_ph, ch->phe_off,
              [&](long long, long long e, uint32_t *code) {
                  const int d = ch->phe_dst[e], s = ch->phe_src[e];
                  if (d < 0 || d >= nc || s < 0 || s >= nc) return false;
                  *code = (uint32_t)d | ((uint32_t)s << I.s_bits);
                  return true;
              },
              [&](long long g) { return (long long)nc + g; }, I.phe_cnt, I.phe_plen, I.phe_off, I.phe_idx, I.phe_W,
              ch->phe_W);
    if (rc) return rc;
    I.pp_cnt.clear();
    I.pp_off.assign(1, 0);
    I.pp_off_dev.release();
    I.pp_idx.release();
    I.pp_W.release();
    if (I.M > 0) {
        if (!ch->pp_off) return fail(ctx, RTBTE_E_INVALID_ARG, "prebuilt ph-ph list required");
        rc = pack(2 * I.M, ch->pp_off,
                  [&](long long, long long e, uint32_t *code) {
                      const int b = ch->pp_b[e], c = ch->pp_c[e];
                      if (b < 0 || b >= I.M || c < 0 || c >= I.M) return false;
                      *code = (uint32_t)b | ((uint32_t)c << I.pp_bits);
                      return true;
                  },
                  [&](long long g) { return (long long)nc + (long long)I.pp_full[g / 2]; }, I.pp_cnt, I.pp_plen,
                  I.pp_off, I.pp_idx, I.pp_W, ch->pp_W);
        if (rc) return rc;
    }
    I.has_channels = true;
    I.counted = true;
    return RTBTE_OK;
}

template <class R>
int download(rtbte_ctx *ctx, InstHost &I, unsigned which, int64_t *off, int32_t *a, int32_t *b, double *W) {
    const std::vector<long long> *po, *cn;
    const DevBuf *di, *dw;
    if (which == RTBTE_EPH) { po = &I.eph_off; cn = &I.eph_cnt; di = &I.eph_idx; dw = &I.eph_W; }
    else if (which == RTBTE_PHE) { po = &I.phe_off; cn = &I.phe_cnt; di = &I.phe_idx; dw = &I.phe_W; }
    else if (which == RTBTE_PHPH) { po = &I.pp_off; cn = &I.pp_cnt; di = &I.pp_idx; dw = &I.pp_W; }
    else return fail(ctx, RTBTE_E_INVALID_ARG, "which must be RTBTE_EPH, RTBTE_PHE or RTBTE_PHPH");
    const long long nseg = (long long)cn->size();
    const long long E = nseg ? (*po)[nseg] : 0;
    std::vector<uint32_t> hidx(E);
    std::vector<R> hW(E);
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (E) {
        RT_CUDA(ctx, cudaMemcpy(hidx.data(), di->p, E * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        RT_CUDA(ctx, cudaMemcpy(hW.data(), dw->p, E * sizeof(R), cudaMemcpyDeviceToHost));
    }
    const uint32_t smask = (1u << I.s_bits) - 1u, pmask = I.pp_bits ? (1u << I.pp_bits) - 1u : 0u;
    long long o = 0;
    off[0] = 0;
    if (which == RTBTE_EPH && I.eph_nqb > 1) {
        // q-blocked e-ph lists: merge each (mode, electron, process) segment's block sub-lists
        // back into one list in ascending source order (a source occurs once per segment)
        const long long nc = I.d.n_c, nqb = I.eph_nqb;
        std::vector<std::pair<uint32_t, long long>> tmp;
        for (long long nu = 0; nu < I.d.nmodes; ++nu)
            for (long long d = 0; d < nc; ++d)
                for (int proc = 0; proc < 2; ++proc) {
                    tmp.clear();
                    for (long long qb = 0; qb < nqb; ++qb) {
                        const long long g = ((nu * nqb + qb) * nc + d) * 2 + proc;
                        for (long long k = 0; k < (*cn)[g]; ++k) tmp.push_back({hidx[(*po)[g] + k], (*po)[g] + k});
                    }
                    std::sort(tmp.begin(), tmp.end(), [&](const std::pair<uint32_t, long long> &x,
                                                          const std::pair<uint32_t, long long> &y) {
                        return (x.first & smask) < (y.first & smask);
                    });
                    for (const auto &t : tmp) {
                        a[o] = (int32_t)(t.first & smask);
                        b[o] = (int32_t)(nu * I.N_q + (t.first >> I.s_bits));
                        W[o] = (double)hW[t.second];
                        ++o;
                    }
                    off[(nu * nc + d) * 2 + proc + 1] = o;
                }
        return RTBTE_OK;
    }
    std::vector<long long> ord;
    std::vector<int32_t> ta, tb;
    std::vector<double> tw;
    for (long long g = 0; g < nseg; ++g) {
        const long long o0 = o;
        for (long long k = 0; k < (*cn)[g]; ++k) {
            const uint32_t e = hidx[(*po)[g] + k];
            if (which == RTBTE_EPH) {
                const int nu = (int)(g / (2LL * I.eph_nqb * I.d.n_c));
                a[o] = (int32_t)(e & smask);
                b[o] = (int32_t)((long long)nu * I.N_q + (e >> I.s_bits));
            } else if (which == RTBTE_PHE) {
                a[o] = (int32_t)(e & smask);
                b[o] = (int32_t)(e >> I.s_bits);
            } else {
                a[o] = (int32_t)(e & pmask);
                b[o] = (int32_t)(e >> I.pp_bits);
            }
            W[o] = (double)hW[(*po)[g] + k];
            ++o;
        }
        // stored blocks are in bank-aware order: hand the segment back sorted by (a, b)
        const long long n = o - o0;
        if (n > 1) {
            ord.resize(n);
            for (long long i = 0; i < n; ++i) ord[i] = o0 + i;
            std::sort(ord.begin(), ord.end(), [&](long long x, long long y) {
                return a[x] != a[y] ? a[x] < a[y] : b[x] < b[y];
            });
            ta.resize(n);
            tb.resize(n);
            tw.resize(n);
            for (long long i = 0; i < n; ++i) {
                ta[i] = a[ord[i]];
                tb[i] = b[ord[i]];
                tw[i] = W[ord[i]];
            }
            for (long long i = 0; i < n; ++i) {
                a[o0 + i] = ta[i];
                b[o0 + i] = tb[i];
                W[o0 + i] = tw[i];
            }
        }
        off[g + 1] = o;
    }
    return RTBTE_OK;
}

// Segments [s0, s1) of the download order (e-ph (mode, electron, process), ph-e phonon, ph-ph
// (sub-lattice phonon, process)), each copied from the device on its own and sorted by (a, b).
template <class R>
int download_range(rtbte_ctx *ctx, InstHost &I, unsigned which, long long s0, long long s1, int64_t *off, int32_t *a,
                   int32_t *b, double *W, long long cap) {
    const std::vector<long long> *po, *cn;
    const DevBuf *di, *dw;
    long long nseg;
    if (which == RTBTE_EPH) { po = &I.eph_off; cn = &I.eph_cnt; di = &I.eph_idx; dw = &I.eph_W; nseg = 2LL * I.d.nmodes * I.d.n_c; }
    else if (which == RTBTE_PHE) { po = &I.phe_off; cn = &I.phe_cnt; di = &I.phe_idx; dw = &I.phe_W; nseg = I.n_ph; }
    else if (which == RTBTE_PHPH) { po = &I.pp_off; cn = &I.pp_cnt; di = &I.pp_idx; dw = &I.pp_W; nseg = 2 * I.M; }
    else return fail(ctx, RTBTE_E_INVALID_ARG, "which must be RTBTE_EPH, RTBTE_PHE or RTBTE_PHPH");
    if (s0 < 0 || s1 < s0 || s1 > nseg) return fail(ctx, RTBTE_E_INVALID_ARG, "segment range out of bounds");
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const uint32_t smask = (1u << I.s_bits) - 1u, pmask = I.pp_bits ? (1u << I.pp_bits) - 1u : 0u;
    const long long nc = I.d.n_c, nqb = which == RTBTE_EPH ? std::max(I.eph_nqb, 1) : 1;
    std::vector<uint32_t> hidx;
    std::vector<R> hW;
    std::vector<std::pair<std::pair<int32_t, int32_t>, double>> seg;
    long long o = 0;
    off[0] = 0;
    for (long long g = s0; g < s1; ++g) {
        seg.clear();
        for (long long qb = 0; qb < nqb; ++qb) {
            long long sg = g;
            if (which == RTBTE_EPH) sg = (((g / (2 * nc)) * nqb + qb) * nc + (g / 2) % nc) * 2 + g % 2;
            const long long n = (*cn)[sg], at = (*po)[sg];
            if (n == 0) continue;
            hidx.resize(n);
            hW.resize(n);
            RT_CUDA(ctx, cudaMemcpy(hidx.data(), di->as<uint32_t>() + at, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
            RT_CUDA(ctx, cudaMemcpy(hW.data(), dw->as<R>() + at, n * sizeof(R), cudaMemcpyDeviceToHost));
            for (long long k = 0; k < n; ++k) {
                const uint32_t e = hidx[k];
                int32_t x, y;
                if (which == RTBTE_EPH) {
                    x = (int32_t)(e & smask);
                    y = (int32_t)((g / (2 * nc)) * I.N_q + (e >> I.s_bits));
                } else if (which == RTBTE_PHE) {
                    x = (int32_t)(e & smask);
                    y = (int32_t)(e >> I.s_bits);
                } else {
                    x = (int32_t)(e & pmask);
                    y = (int32_t)(e >> I.pp_bits);
                }
                seg.push_back({{x, y}, (double)hW[k]});
            }
        }
        std::sort(seg.begin(), seg.end(), [](const auto &p, const auto &q) { return p.first < q.first; });
        if (a) {
            if (o + (long long)seg.size() > cap) return fail(ctx, RTBTE_E_INVALID_ARG, "entry arrays too small");
            for (const auto &t : seg) {
                a[o] = t.first.first;
                b[o] = t.first.second;
                W[o] = t.second;
                ++o;
            }
        } else {
            o += (long long)seg.size();
        }
        off[g - s0 + 1] = o;
    }
    return RTBTE_OK;
}

int ensure_plan(rtbte_ctx *ctx) {
    for (auto &I : ctx->inst)
        if (!I.has_channels) return fail(ctx, RTBTE_E_STATE, "an instance has no channels (call rtbte_upload_channels)");
    if (!ctx->plan_valid) return make_plan(ctx);
    return RTBTE_OK;
}

}  // namespace
}  // namespace rtbte

using namespace rtbte;

extern "C" {

void rtbte_desc_defaults(rtbte_desc *d) {
    if (!d) return;
    std::memset(d, 0, sizeof(*d));
    d->n_instances = 1;
    d->precision = RTBTE_PREC_FP32_COMP;
    d->hbar = 6.582119569e-4;
}

void rtbte_integ_defaults(rtbte_integ *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->method = RTBTE_ZON43;
    o->fast_method = RTBTE_ZON43;
    o->rtol = 1e-5;
    o->atol_c = 1e-9;
    o->atol_ph = 1e-12;
    o->a1 = 0.58;
    o->a2 = 0.21;
    o->a3 = 0.1;
    o->safety = 0.96;
    o->growth = 20.0;
    o->growth_first = 1e4;
    o->etamxf = 0.3;
    o->etamin = 0.1;
    o->small_nef = 2;
    o->max_nef = 7;
}

int rtbte_create(const rtbte_desc *d, rtbte_ctx **out) {
    if (!d || !out || d->n_instances < 1 || !d->inst || !(d->hbar > 0) ||
        (d->precision != RTBTE_PREC_FP32_COMP && d->precision != RTBTE_PREC_FP64) || d->eph_q_blocks < 0 ||
        d->eph_q_blocks > 256)
        return RTBTE_E_INVALID_ARG;
    *out = nullptr;
    rtbte_ctx *ctx = new (std::nothrow) rtbte_ctx();
    if (!ctx) return RTBTE_E_OOM;
    int rc = RTBTE_OK;
    auto bail = [&](int code) {
        rtbte_destroy(ctx);
        return code;
    };
    ctx->device = d->device;
    ctx->precision = d->precision;
    ctx->eph_q_blocks = d->eph_q_blocks;
    ctx->real_size = d->precision == RTBTE_PREC_FP64 ? 8 : 4;
    ctx->hbar = d->hbar;
    ctx->stream = reinterpret_cast<cudaStream_t>(d->stream);
    if (cudaSetDevice(d->device) != cudaSuccess) return bail(cuda_fail(ctx, cudaErrorInvalidDevice, "cudaSetDevice"));
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d->device) != cudaSuccess)
        return bail(cuda_fail(ctx, cudaErrorInvalidDevice, "cudaDeviceGetAttribute"));
    ctx->num_sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, d->device) != cudaSuccess)
        return bail(cuda_fail(ctx, cudaErrorInvalidDevice, "cudaDeviceGetAttribute"));
    ctx->smem_optin = (size_t)v;
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(cuda_fail(ctx, cudaErrorUnknown, "cudaStreamCreate"));
    ctx->inst.resize(d->n_instances);
    long long y = 0, f = 0, N = 0, P = 0;
    for (int i = 0; i < d->n_instances; ++i) {
        InstHost &I = ctx->inst[i];
        if ((rc = setup_instance(ctx, d->inst[i], I))) return bail(rc);
        I.y_off = y;
        I.f_off = f;
        I.N_off = N;
        I.P_off = P;
        y += I.d.n_c + I.n_ph;
        f += I.n_c_pad;
        N += (long long)I.d.nmodes * I.N_q_pad;
        P += I.M_pad;
    }
    ctx->n_y = y;
    if (d->row_end > d->row_begin || d->row_begin != 0 || d->row_end != 0) {  // a row slice
        if (d->n_instances != 1 || d->row_begin < 0 || d->row_end <= d->row_begin || d->row_end > y)
            return bail(fail(ctx, RTBTE_E_INVALID_ARG, "row slice must lie in [0, n_y) of a single-instance context"));
        ctx->inst[0].row_lo = d->row_begin;
        ctx->inst[0].row_hi = d->row_end;
        ctx->sliced = true;
    } else {
        for (auto &I : ctx->inst) {
            I.row_lo = 0;
            I.row_hi = I.d.n_c + I.n_ph;
        }
    }
    ctx->popf_len = f;
    ctx->popN_len = N;
    ctx->popP_len = P;
    const size_t R = ctx->real_size;
    if ((rc = dev_alloc(ctx, ctx->popf, R * (f + 4), true)) || (rc = dev_alloc(ctx, ctx->popN, R * (N + 4), true)) ||
        (rc = dev_alloc(ctx, ctx->popP, R * (P + 4), true)) ||
        (rc = dev_alloc(ctx, ctx->Y[0], sizeof(double) * y, true)) ||
        (rc = dev_alloc(ctx, ctx->Y[1], sizeof(double) * y, true)) ||
        (rc = dev_alloc(ctx, ctx->K, sizeof(double) * y * kMaxStages, true)) ||
        (rc = dev_alloc(ctx, ctx->Fs, sizeof(double) * y * 3, true)) ||
        (rc = dev_alloc(ctx, ctx->forcing, sizeof(double) * y, true)) ||
        (rc = dev_alloc(ctx, ctx->wrms_part, sizeof(double) * (2 * y + 2LL * kWrmsChunks * d->n_instances), true)) ||
        (rc = dev_alloc(ctx, ctx->ctl, sizeof(Ctl) * d->n_instances, true)) ||
        (rc = dev_alloc(ctx, ctx->range_scratch, sizeof(unsigned long long) * d->n_instances, true)))
        return bail(rc);
    if (cudaMallocHost(&ctx->ctl_host, sizeof(Ctl) * d->n_instances) != cudaSuccess)
        return bail(cuda_fail(ctx, cudaErrorMemoryAllocation, "cudaMallocHost"));
    std::memset(ctx->ctl_host, 0, sizeof(Ctl) * d->n_instances);
    for (int i = 0; i < d->n_instances; ++i)
        if ((rc = upload_tables(ctx, i))) return bail(rc);
    *out = ctx;
    return RTBTE_OK;
}

int rtbte_upload_channels(rtbte_ctx *ctx, int inst, const rtbte_channels *ch) {
    Range nvtx_range("rtbte_upload_channels");
    if (!ctx) return RTBTE_E_INVALID_ARG;
    if (!ch || inst < 0 || inst >= (int)ctx->inst.size()) return fail(ctx, RTBTE_E_INVALID_ARG, "bad instance or channels");
    InstHost &I = ctx->inst[inst];
    ctx->plan_valid = false;
    I.has_channels = false;
    I.counted = false;
    destroy_graphs(ctx);  // graphs capture the plan's pointers
    if (ch->mode == RTBTE_CH_BUILD) return build_channels(ctx, inst, false);
    if (ch->mode == RTBTE_CH_COUNT) return build_channels(ctx, inst, true);
    if (ch->mode == RTBTE_CH_PREBUILT)
        return ctx->precision == RTBTE_PREC_FP64 ? upload_prebuilt<double>(ctx, I, ch) : upload_prebuilt<float>(ctx, I, ch);
    return fail(ctx, RTBTE_E_INVALID_ARG, "unknown channel mode");
}

int rtbte_rhs(rtbte_ctx *ctx, double t, const double *y, double *ydot, unsigned parts) {
    Range nvtx_range("rtbte_rhs");
    (void)t;
    if (!ctx) return RTBTE_E_INVALID_ARG;
    if (!y || !ydot || parts == 0 || parts > RTBTE_ALL) return fail(ctx, RTBTE_E_INVALID_ARG, "bad rhs arguments");
    int rc;
    if ((rc = ensure_plan(ctx))) return rc;
    const bool dy = ptr_is_device(y), dd = ptr_is_device(ydot);
    if (dy != dd) return fail(ctx, RTBTE_E_INVALID_ARG, "y and ydot must both be device or both be host pointers");
    if (dy) {
        if ((rc = launch_prep_from_y(ctx, y, ctx->stream))) return rc;
        if ((rc = launch_rhs_core(ctx, parts, nullptr, ctx->stream))) return rc;
        return launch_rows(ctx, parts, ydot, nullptr, ctx->stream);
    }
    const size_t nb = sizeof(double) * ctx->n_y;
    if (!ctx->ystage.p && (rc = dev_alloc(ctx, ctx->ystage, nb, false))) return rc;
    if (!ctx->ydstage.p && (rc = dev_alloc(ctx, ctx->ydstage, nb, false))) return rc;
    RT_CUDA(ctx, cudaMemcpyAsync(ctx->ystage.p, y, nb, cudaMemcpyHostToDevice, ctx->stream));
    if ((rc = launch_prep_from_y(ctx, ctx->ystage.as<double>(), ctx->stream))) return rc;
    if ((rc = launch_rhs_core(ctx, parts, nullptr, ctx->stream))) return rc;
    if ((rc = launch_rows(ctx, parts, ctx->ydstage.as<double>(), nullptr, ctx->stream))) return rc;
    RT_CUDA(ctx, cudaMemcpyAsync(ydot, ctx->ydstage.p, nb, cudaMemcpyDeviceToHost, ctx->stream));
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RTBTE_OK;
}

int rtbte_get_controller(const rtbte_ctx *ctx, int inst, rtbte_controller *out) {
    if (!ctx || !out || inst < 0 || inst >= (int)ctx->inst.size()) return RTBTE_E_INVALID_ARG;
    const Ctl &c = ctx->ctl_host[inst];
    out->t = c.t;
    out->h = c.h;
    out->eps1 = c.eps1;
    out->eps2 = c.eps2;
    out->first = c.first;
    out->nef = c.nef;
    return RTBTE_OK;
}

int rtbte_set_controller(rtbte_ctx *ctx, int inst, const rtbte_controller *in) {
    if (!ctx || !in || inst < 0 || inst >= (int)ctx->inst.size()) return RTBTE_E_INVALID_ARG;
    if (!(in->h >= 0) || !(in->eps1 > 0) || !(in->eps2 > 0)) return fail(ctx, RTBTE_E_INVALID_ARG, "bad controller state");
    Ctl &c = ctx->ctl_host[inst];
    c.t = in->t;
    c.h = in->h;
    c.eps1 = in->eps1;
    c.eps2 = in->eps2;
    c.first = in->first;
    c.nef = in->nef;
    return RTBTE_OK;
}

int rtbte_phph_rates(rtbte_ctx *ctx, const double *y, double *rates) {
    Range nvtx_range("rtbte_phph_rates");
    if (!ctx) return RTBTE_E_INVALID_ARG;
    if (!y || !rates || !ptr_is_device(y) || !ptr_is_device(rates))
        return fail(ctx, RTBTE_E_INVALID_ARG, "y and rates must be device pointers");
    int rc;
    if ((rc = ensure_plan(ctx))) return rc;
    RT_CUDA(ctx, cudaMemsetAsync(rates, 0, sizeof(double) * ctx->n_y, ctx->stream));
    if ((rc = launch_prep_from_y(ctx, y, ctx->stream))) return rc;
    for (int i = 0; i < (int)ctx->inst.size(); ++i)
        if ((rc = launch_pp_rates(ctx, i, rates, ctx->stream))) return rc;
    return RTBTE_OK;
}

int rtbte_advance_to(rtbte_ctx *ctx, double t_out, double *y, const rtbte_integ *opt, rtbte_stats *st) {
    Range nvtx_range("rtbte_advance_to");
    if (!ctx) return RTBTE_E_INVALID_ARG;
    if (!y || !opt) return fail(ctx, RTBTE_E_INVALID_ARG, "bad advance_to arguments");
    if (ctx->sliced)
        return fail(ctx, RTBTE_E_STATE, "a row-sliced context evaluates its rows only; integrate the gathered RHS");
    int rc;
    if ((rc = ensure_plan(ctx))) return rc;
    if (ptr_is_device(y)) return advance_to(ctx, t_out, y, opt, st);
    // host state: staged through a context buffer (copy in, integrate, copy the result back)
    const size_t nb = sizeof(double) * ctx->n_y;
    if (!ctx->ystage.p && (rc = dev_alloc(ctx, ctx->ystage, nb, false))) return rc;
    RT_CUDA(ctx, cudaMemcpyAsync(ctx->ystage.p, y, nb, cudaMemcpyHostToDevice, ctx->stream));
    const int status = advance_to(ctx, t_out, ctx->ystage.as<double>(), opt, st);
    if (status == RTBTE_E_CUDA || status == RTBTE_E_INVALID_ARG || status == RTBTE_E_OOM || status == RTBTE_E_STATE)
        return status;  // y untouched
    RT_CUDA(ctx, cudaMemcpyAsync(y, ctx->ystage.p, nb, cudaMemcpyDeviceToHost, ctx->stream));
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return status;
}

int rtbte_get_sizes(const rtbte_ctx *ctx, int inst, rtbte_sizes *out) {
    if (!ctx || !out || inst < 0 || inst >= (int)ctx->inst.size()) return RTBTE_E_INVALID_ARG;
    const InstHost &I = ctx->inst[inst];
    std::memset(out, 0, sizeof(*out));
    out->n_c = I.d.n_c;
    out->n_ph = I.n_ph;
    out->n_pp = I.M;
    out->y_offset = I.y_off;
    out->n_y_total = ctx->n_y;
    auto sum = [](const std::vector<long long> &v) {
        long long s = 0;
        for (long long x : v) s += x;
        return s;
    };
    out->eph_entries = sum(I.eph_cnt);
    out->phe_entries = sum(I.phe_cnt);
    out->pp_entries = sum(I.pp_cnt);
    out->eph_stored = I.eph_off.empty() ? 0 : I.eph_off.back();
    out->phe_stored = I.phe_off.empty() ? 0 : I.phe_off.back();
    out->pp_stored = I.pp_off.empty() ? 0 : I.pp_off.back();
    out->work_items = ctx->n_items;
    const long long es = 4 + (long long)ctx->real_size;
    out->channel_bytes = es * (out->eph_stored + out->phe_stored + out->pp_stored);
    out->eph_q_blocks = I.has_channels ? I.eph_nqb : 0;
    return RTBTE_OK;
}

int rtbte_row_entries(const rtbte_ctx *ctx, int inst, int64_t *counts) {
    if (!ctx || !counts || inst < 0 || inst >= (int)ctx->inst.size()) return RTBTE_E_INVALID_ARG;
    const InstHost &I = ctx->inst[inst];
    if (!I.counted) return RTBTE_E_STATE;
    const long long nc = I.d.n_c;
    std::fill(counts, counts + nc + I.n_ph, (int64_t)0);
    for (size_t g = 0; g < I.eph_cnt.size(); ++g) counts[(g / 2) % nc] += I.eph_cnt[g];  // (mode, block, d, proc)
    for (size_t p = 0; p < I.phe_cnt.size(); ++p) counts[nc + p] += I.phe_cnt[p];
    for (size_t g = 0; g < I.pp_cnt.size(); ++g) counts[nc + I.pp_full[g / 2]] += I.pp_cnt[g];
    return RTBTE_OK;
}

int rtbte_download_channels(rtbte_ctx *ctx, int inst, unsigned which, int64_t *off, int32_t *a, int32_t *b, double *W) {
    if (!ctx) return RTBTE_E_INVALID_ARG;
    if (inst < 0 || inst >= (int)ctx->inst.size() || !off || !a || !b || !W)
        return fail(ctx, RTBTE_E_INVALID_ARG, "bad download arguments");
    InstHost &I = ctx->inst[inst];
    if (!I.has_channels) return fail(ctx, RTBTE_E_STATE, "instance has no channels");
    return ctx->precision == RTBTE_PREC_FP64 ? download<double>(ctx, I, which, off, a, b, W)
                                             : download<float>(ctx, I, which, off, a, b, W);
}

int rtbte_download_segments(rtbte_ctx *ctx, int inst, unsigned which, int64_t seg_begin, int64_t seg_end, int64_t *off,
                            int32_t *a, int32_t *b, double *W, int64_t cap) {
    if (!ctx) return RTBTE_E_INVALID_ARG;
    if (inst < 0 || inst >= (int)ctx->inst.size() || !off || (a && (!b || !W)))
        return fail(ctx, RTBTE_E_INVALID_ARG, "bad download arguments");
    InstHost &I = ctx->inst[inst];
    if (!I.has_channels) return fail(ctx, RTBTE_E_STATE, "instance has no channels");
    return ctx->precision == RTBTE_PREC_FP64
               ? download_range<double>(ctx, I, which, seg_begin, seg_end, off, a, b, W, cap)
               : download_range<float>(ctx, I, which, seg_begin, seg_end, off, a, b, W, cap);
}

int rtbte_set_stream(rtbte_ctx *ctx, void *stream) {
    if (!ctx) return RTBTE_E_INVALID_ARG;
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    return RTBTE_OK;
}

int rtbte_autotune(rtbte_ctx *ctx, unsigned parts, int *chosen) {
    Range nvtx_range("rtbte_autotune");
    if (!ctx) return RTBTE_E_INVALID_ARG;
    if (parts == 0 || parts > RTBTE_ALL) return fail(ctx, RTBTE_E_INVALID_ARG, "bad parts");
    int rc;
    if ((rc = ensure_plan(ctx))) return rc;
    destroy_graphs(ctx);  // graphs keep the previous split's table pointer
    return autotune(ctx, parts, chosen);
}

int rtbte_get_tuning(const rtbte_ctx *ctx, int32_t *item_weight, int32_t *prefetch_items, double *static_share) {
    if (!ctx) return RTBTE_E_INVALID_ARG;
    const rtbte::LaunchTuning &L = ctx->lt[RTBTE_ALL];
    if (item_weight) *item_weight = L.w;
    if (prefetch_items) *prefetch_items = L.pf;
    if (static_share) *static_share = L.sf;
    return RTBTE_OK;
}

int rtbte_set_graph_mode(rtbte_ctx *ctx, int use_graphs) {
    if (!ctx) return RTBTE_E_INVALID_ARG;
    ctx->use_graphs = use_graphs != 0;
    return RTBTE_OK;
}

int rtbte_set_kernel_timing(rtbte_ctx *ctx, int enable) {
    if (!ctx) return RTBTE_E_INVALID_ARG;
    ctx->timing = enable != 0;
    return RTBTE_OK;
}

int rtbte_kernel_time(rtbte_ctx *ctx, double *total_ms, int64_t *launches) {
    if (!ctx || !total_ms || !launches) return RTBTE_E_INVALID_ARG;
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double tot = 0.0;
    for (auto &pr : ctx->ev_pending) {
        float ms = 0.f;
        RT_CUDA(ctx, cudaEventElapsedTime(&ms, pr.first, pr.second));
        tot += ms;
        ctx->ev_pool.push_back(pr.first);
        ctx->ev_pool.push_back(pr.second);
    }
    *total_ms = tot;
    *launches = (int64_t)ctx->ev_pending.size();
    ctx->ev_pending.clear();
    return RTBTE_OK;
}

int64_t rtbte_launch_count(const rtbte_ctx *ctx) { return ctx ? ctx->launches : 0; }

const char *rtbte_last_error(const rtbte_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

const char *rtbte_status_string(int s) {
    switch (s) {
        case RTBTE_OK: return "ok";
        case RTBTE_E_INVALID_ARG: return "invalid argument";
        case RTBTE_E_OOM: return "out of memory";
        case RTBTE_E_CUDA: return "CUDA error";
        case RTBTE_E_TOO_MANY_STEPS: return "too many steps";
        case RTBTE_E_STEP_UNDERFLOW: return "step size underflow";
        case RTBTE_E_ERR_TEST_FAIL: return "repeated error-test failures";
        case RTBTE_E_NONFINITE: return "non-finite value";
        case RTBTE_E_TIMEOUT: return "device wait timed out";
        case RTBTE_E_STATE: return "call out of order";
        case RTBTE_E_UNSUPPORTED: return "unsupported size";
        default: return "unknown status";
    }
}

void rtbte_destroy(rtbte_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    sur_orphan(ctx);
    destroy_graphs(ctx);
    ctx->loop_iter.release();
    if (ctx->loop_iter_host) cudaFreeHost(ctx->loop_iter_host);
    ctx->loop_iter_host = nullptr;
    for (auto &I : ctx->inst) {
        DevBuf *bufs[] = {&I.t_ek, &I.t_eps, &I.t_eid, &I.t_eidinv, &I.t_omega, &I.t_kmap, &I.t_lut, &I.t_g2,
                          &I.t_ppfull, &I.t_ppinv, &I.eph_idx, &I.eph_W, &I.phe_idx, &I.phe_W, &I.pp_idx, &I.pp_W,
                          &I.pp_off_dev};
        for (DevBuf *b : bufs) b->release();
    }
    ctx->tail_tab.release();
    ctx->tail_ctr.release();
    DevBuf *bufs[] = {&ctx->popf, &ctx->popN, &ctx->popP, &ctx->instdev, &ctx->compact, &ctx->items, &ctx->groups,
                      &ctx->partials, &ctx->rowoff, &ctx->rowmid, &ctx->cta_tab, &ctx->gwt, &ctx->dyn_tab, &ctx->Y[0], &ctx->Y[1],
                      &ctx->K, &ctx->Fs, &ctx->forcing, &ctx->wrms_part, &ctx->ctl, &ctx->ystage, &ctx->ydstage,
                      &ctx->range_scratch, &ctx->slow_save};
    for (DevBuf *b : bufs) b->release();
    for (auto &pr : ctx->ev_pending) {
        ctx->ev_pool.push_back(pr.first);
        ctx->ev_pool.push_back(pr.second);
    }
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->ctl_host) cudaFreeHost(ctx->ctl_host);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
}

}  // extern "C"
