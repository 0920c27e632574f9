// rhs.cu -- the collision-integral kernels (Eq. e-ph, Eq. ph-ph) and their execution plan.
//
// One persistent launch evaluates the selected parts of the RHS for every instance.  The
// stored channel entries are streamed from HBM exactly once per evaluation (16-byte
// cache-streaming loads, 4 entries per lane), while the populations they gather are
// staged per CTA in shared memory: the instance's electron occupations f plus, for e-ph
// work, the occupations N of one phonon mode (the e-ph lists are blocked by mode for this
// reason); for ph-e work only f; for ph-ph work the sub-lattice N.  Each warp owns one
// work item (<= 512 entries of a single destination segment) and reduces it with a
// compensated (two-sum) accumulation and a compensated warp-shuffle tree; the partial is
// written per item, and the row kernels add partials in item order (deterministic).
//
// Per-entry arithmetic uses the exact algebraic reductions of the paper's factors
// (Methods A):  F_em = f(1-f') + N(f-f'),  F_abs = N(f-f') - f'(1-f),
//               G_em = N(N'+N''+1) - N'N'',  G_abs = N(N''-N') - N'(N''+1).
#include <algorithm>
#include <cstring>
#include <numeric>

#include "internal.cuh"
#include "rows.cuh"

namespace rtbte {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kItemOverhead = 24;  // scheduling weight of an item beyond its entries

template <class R> __device__ __forceinline__ R Fem(R f, R fp, R N) { return f * (R(1) - fp) + N * (f - fp); }
template <class R> __device__ __forceinline__ R Fab(R f, R fp, R N) { return N * (f - fp) - fp * (R(1) - f); }
template <class R> __device__ __forceinline__ R Gem(R Na, R Nb, R Nc) { return Na * (Nb + Nc + R(1)) - Nb * Nc; }
template <class R> __device__ __forceinline__ R Gab(R Na, R Nb, R Nc) { return Na * (Nc - Nb) - Nb * (Nc + R(1)); }

// s + c += x with the rounding error of the addition kept in c (Knuth two-sum).
template <class R> __device__ __forceinline__ void two_sum(R &s, R &c, R x) {
    R t = s + x;
    R bp = t - s;
    R e = (s - (t - bp)) + (x - bp);
    s = t;
    c += e;
}

// Compensated butterfly reduction; every lane ends with the same bits.
template <class R> __device__ __forceinline__ void warp_reduce2(R &s, R &c) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        R s2 = __shfl_xor_sync(kFull, s, o);
        R c2 = __shfl_xor_sync(kFull, c, o);
        R t = s + s2;
        R bp = t - s;
        R e = (s - (t - bp)) + (s2 - bp);
        s = t;
        c = (c + c2) + e;
    }
}

template <class R> struct W4;
template <> struct W4<float> {
    static __device__ __forceinline__ void load(const void *W, long long v, float w[4]) {
        float4 x = __ldcs(reinterpret_cast<const float4 *>(W) + v);
        w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
    }
};
template <> struct W4<double> {
    static __device__ __forceinline__ void load(const void *W, long long v, double w[4]) {
        double2 a = __ldcs(reinterpret_cast<const double2 *>(W) + 2 * v);
        double2 b = __ldcs(reinterpret_cast<const double2 *>(W) + 2 * v + 1);
        w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
    }
};

struct KParams {
    const Item *items;
    const Group *groups;
    int n_groups;
    const int *cta_v;  // [grid+1] virtual item starts for this part mask
    int rv[3], ri[3], rlen[3];
    int nranges;
    void *partials;
    const void *popf, *popN, *popP;
    const Ctl *ctl;  // launches inside an integrator skip when the integration is done
};

template <class R>
__device__ __forceinline__ void stage_copy(R *dst, const R *src, int n) {
    const int nvec = (int)((long long)n * sizeof(R) / 16);
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(dst);
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
        const char *g = reinterpret_cast<const char *>(src) + 16LL * i;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sbase + 16u * i), "l"(g) : "memory");
    }
}

template <class R, bool STAGED>
__device__ __forceinline__ void run_item(const KParams &P, const Group &G, int iid, const R *s0, const R *s1, int lane) {
    const Item it = P.items[iid];
    const int nv = it.len >> 2;
    const uint4 *ip = reinterpret_cast<const uint4 *>(G.idx + it.begin);
    const long long wv0 = it.begin >> 2;
    uint4 iv[4];
    R wv[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int v = lane + 32 * j;
        if (v < nv) {
            iv[j] = __ldcs(ip + v);
            W4<R>::load(G.W, wv0 + v, wv[j]);
        }
    }
    R acc = R(0), cmp = R(0);
    if (G.part == PART_EPH) {
        const unsigned smask = (1u << G.s_bits) - 1u;
        const R fd = s0[it.dest];
        // s0 = f of the instance, s1 = N of this mode
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (lane + 32 * j < nv) {
                const unsigned e[4] = {iv[j].x, iv[j].y, iv[j].z, iv[j].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const R fs = s0[e[k] & smask];
                    const R N = s1[e[k] >> G.s_bits];
                    const R F = it.proc ? Fab(fd, fs, N) : Fem(fd, fs, N);
                    two_sum(acc, cmp, wv[j][k] * F);
                }
            }
        }
    } else if (G.part == PART_PHE) {
        const unsigned smask = (1u << G.s_bits) - 1u;
        const R Np = reinterpret_cast<const R *>(P.popN)[G.N_inst + it.dest];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (lane + 32 * j < nv) {
                const unsigned e[4] = {iv[j].x, iv[j].y, iv[j].z, iv[j].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const R fd = s0[e[k] & smask];
                    const R fs = s0[e[k] >> G.s_bits];
                    two_sum(acc, cmp, wv[j][k] * Fab(fd, fs, Np));
                }
            }
        }
    } else {
        const unsigned pmask = (1u << G.pp_bits) - 1u;
        const R Na = s0[it.dest];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (lane + 32 * j < nv) {
                const unsigned e[4] = {iv[j].x, iv[j].y, iv[j].z, iv[j].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const R Nb = s0[e[k] & pmask];
                    const R Nc = s0[e[k] >> G.pp_bits];
                    const R Gv = it.proc ? Gab(Na, Nb, Nc) : Gem(Na, Nb, Nc);
                    two_sum(acc, cmp, wv[j][k] * Gv);
                }
            }
        }
    }
    warp_reduce2(acc, cmp);
    if (lane == 0) {
        R *out = reinterpret_cast<R *>(P.partials) + 2LL * iid;
        out[0] = acc;
        out[1] = cmp;
    }
}

template <class R, bool STAGED, int MINB>
__global__ void __launch_bounds__(kRhsThreads, MINB) rhs_kernel(KParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (P.ctl && P.ctl->done) return;
    R *sm = reinterpret_cast<R *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int v0 = P.cta_v[blockIdx.x], v1 = P.cta_v[blockIdx.x + 1];
    for (int r = 0; r < P.nranges; ++r) {
        const int a = max(v0, P.rv[r]), b = min(v1, P.rv[r] + P.rlen[r]);
        if (a >= b) continue;
        const int ra = P.ri[r] + (a - P.rv[r]), rb = ra + (b - a);
        int lo = 0, hi = P.n_groups - 1;  // last group with item_begin <= ra
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (P.groups[mid].item_begin <= ra) lo = mid; else hi = mid - 1;
        }
        for (int g = lo; g < P.n_groups; ++g) {
            const Group G = P.groups[g];
            if (G.item_begin >= rb) break;
            const int ia = max(ra, G.item_begin), ib = min(rb, G.item_end);
            if (ia >= ib) continue;
            const R *s0, *s1;
            if (STAGED) {
                __syncthreads();  // the previous group's readers are done with the buffer
                const R *src0 = reinterpret_cast<const R *>(G.part == PART_PP ? P.popP : P.popf) + G.stage0_src;
                stage_copy<R>(sm, src0, G.stage0_len);
                if (G.stage1_len > 0)
                    stage_copy<R>(sm + G.stage0_len, reinterpret_cast<const R *>(P.popN) + G.stage1_src, G.stage1_len);
                asm volatile("cp.async.commit_group;\n" ::: "memory");
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                __syncthreads();
                s0 = sm;
                s1 = sm + G.stage0_len;
            } else {
                s0 = reinterpret_cast<const R *>(G.part == PART_PP ? P.popP : P.popf) + G.stage0_src;
                s1 = reinterpret_cast<const R *>(P.popN) + G.stage1_src;
            }
            for (int iid = ia + warp; iid < ib; iid += nwarps) run_item<R, STAGED>(P, G, iid, s0, s1, lane);
        }
    }
}

// y (FP64) -> population copies in the compute precision
template <class R>
__global__ void prep_kernel(RowParams Q, const double *y, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = Q.n_inst > 1 ? find_inst(Q, c) : 0;
        const InstDev I = Q.inst[i];
        write_pops<R>(Q, I, c - I.y_off, y[c]);
    }
}

template <class R>
__global__ void rows_kernel(RowParams Q, unsigned parts, double *out, const double *forcing, long long n) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = Q.n_inst > 1 ? find_inst(Q, c) : 0;
        const InstDev I = Q.inst[i];
        double v = row_value<R>(Q, I, c - I.y_off, parts);
        if (forcing) v += forcing[c];
        out[c] = v;
    }
}

template <class T> int upload_vec(rtbte_ctx *ctx, DevBuf &b, const std::vector<T> &h) {
    b.release();
    size_t bytes = std::max<size_t>(h.size() * sizeof(T), 16);
    RT_CUDA(ctx, cudaMalloc(&b.p, bytes));
    b.bytes = bytes;
    if (!h.empty()) RT_CUDA(ctx, cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return RTBTE_OK;
}

}  // namespace

RowParams row_params(rtbte_ctx *ctx) {
    RowParams Q;
    Q.inst = ctx->instdev.as<InstDev>();
    Q.n_inst = (int)ctx->inst.size();
    Q.eoff = ctx->eoff.as<int>();
    Q.poff = ctx->poff.as<int>();
    Q.ppoff = ctx->ppoff.as<int>();
    Q.compact = ctx->compact.as<int>();
    Q.partials = ctx->partials.p;
    Q.popf = ctx->popf.p;
    Q.popN = ctx->popN.p;
    Q.popP = ctx->popP.p;
    return Q;
}

// Build the work items, staging groups, per-row item offsets and per-CTA work ranges.
int make_plan(rtbte_ctx *ctx) {
    const size_t R = ctx->real_size;
    std::vector<Item> items;
    std::vector<Group> groups;
    std::vector<int> eoff, poff, ppoff;
    std::vector<InstDev> idev(ctx->inst.size());
    auto add_seg = [&](long long b, long long e, int dest, int proc) {
        for (long long x = b; x < e; x += kItemEntries) {
            Item it;
            it.begin = x;
            it.dest = dest;
            it.len = (unsigned short)std::min<long long>(kItemEntries, e - x);
            it.proc = (unsigned char)proc;
            it.pad = 0;
            items.push_back(it);
        }
    };
    size_t max_stage = 0;
    // e-ph groups (instance, mode)
    for (size_t i = 0; i < ctx->inst.size(); ++i) {
        InstHost &I = ctx->inst[i];
        idev[i].eoff_base = (long long)eoff.size();
        for (int nu = 0; nu < I.d.nmodes; ++nu) {
            Group G{};
            G.idx = I.eph_idx.as<uint32_t>();
            G.W = I.eph_W.p;
            G.item_begin = (int)items.size();
            G.part = PART_EPH;
            G.inst = (int)i;
            G.nu = nu;
            G.s_bits = I.s_bits;
            G.n_q_pad = I.N_q_pad;
            G.stage0_len = I.n_c_pad;
            G.stage0_src = I.f_off;
            G.stage1_len = I.N_q_pad;
            G.stage1_src = I.N_off + (long long)nu * I.N_q_pad;
            G.f_inst = I.f_off;
            G.N_inst = I.N_off;
            G.P_inst = I.P_off;
            for (int d = 0; d < I.d.n_c; ++d) {
                eoff.push_back((int)items.size());
                long long g = ((long long)nu * I.d.n_c + d) * 2;
                add_seg(I.eph_off[g], I.eph_off[g + 1], d, 0);
                add_seg(I.eph_off[g + 1], I.eph_off[g + 2], d, 1);
            }
            eoff.push_back((int)items.size());
            G.item_end = (int)items.size();
            groups.push_back(G);
            max_stage = std::max(max_stage, (size_t)(G.stage0_len + G.stage1_len) * R);
        }
    }
    ctx->part_first[PART_EPH] = 0;
    ctx->part_items[PART_EPH] = (int)items.size();
    // ph-e groups (instance)
    for (size_t i = 0; i < ctx->inst.size(); ++i) {
        InstHost &I = ctx->inst[i];
        idev[i].poff_base = (long long)poff.size();
        Group G{};
        G.idx = I.phe_idx.as<uint32_t>();
        G.W = I.phe_W.p;
        G.item_begin = (int)items.size();
        G.part = PART_PHE;
        G.inst = (int)i;
        G.s_bits = I.s_bits;
        G.n_q_pad = I.N_q_pad;
        G.stage0_len = I.n_c_pad;
        G.stage0_src = I.f_off;
        G.f_inst = I.f_off;
        G.N_inst = I.N_off;
        G.P_inst = I.P_off;
        for (long long p = 0; p < I.n_ph; ++p) {
            poff.push_back((int)items.size());
            int nu = (int)(p / I.N_q);
            long long q = p - (long long)nu * I.N_q;
            add_seg(I.phe_off[p], I.phe_off[p + 1], (int)((long long)nu * I.N_q_pad + q), 1);
        }
        poff.push_back((int)items.size());
        G.item_end = (int)items.size();
        groups.push_back(G);
        max_stage = std::max(max_stage, (size_t)G.stage0_len * R);
    }
    ctx->part_first[PART_PHE] = ctx->part_items[PART_EPH];
    ctx->part_items[PART_PHE] = (int)items.size() - ctx->part_first[PART_PHE];
    // ph-ph groups (instance)
    for (size_t i = 0; i < ctx->inst.size(); ++i) {
        InstHost &I = ctx->inst[i];
        idev[i].ppoff_base = (long long)ppoff.size();
        if (I.M == 0) continue;
        Group G{};
        G.idx = I.pp_idx.as<uint32_t>();
        G.W = I.pp_W.p;
        G.item_begin = (int)items.size();
        G.part = PART_PP;
        G.inst = (int)i;
        G.pp_bits = I.pp_bits;
        G.stage0_len = I.M_pad;
        G.stage0_src = I.P_off;
        G.f_inst = I.f_off;
        G.N_inst = I.N_off;
        G.P_inst = I.P_off;
        for (long long a = 0; a < I.M; ++a) {
            ppoff.push_back((int)items.size());
            add_seg(I.pp_off[2 * a], I.pp_off[2 * a + 1], (int)a, 0);
            add_seg(I.pp_off[2 * a + 1], I.pp_off[2 * a + 2], (int)a, 1);
        }
        ppoff.push_back((int)items.size());
        G.item_end = (int)items.size();
        groups.push_back(G);
        max_stage = std::max(max_stage, (size_t)G.stage0_len * R);
    }
    ctx->part_first[PART_PP] = ctx->part_first[PART_PHE] + ctx->part_items[PART_PHE];
    ctx->part_items[PART_PP] = (int)items.size() - ctx->part_first[PART_PP];
    if (items.size() >= (size_t)INT32_MAX) return fail(ctx, RTBTE_E_UNSUPPORTED, "too many work items");
    ctx->n_items = (int)items.size();
    ctx->n_groups = (int)groups.size();
    // instance layout for the row kernels
    std::vector<int> compact;
    for (size_t i = 0; i < ctx->inst.size(); ++i) {
        InstHost &I = ctx->inst[i];
        InstDev &D = idev[i];
        D.y_off = I.y_off;
        D.n_c = I.d.n_c;
        D.n_ph = (int)I.n_ph;
        D.M = (int)I.M;
        D.nmodes = I.d.nmodes;
        D.N_q = (int)I.N_q;
        D.N_q_pad = I.N_q_pad;
        D.f_off = I.f_off;
        D.N_off = I.N_off;
        D.P_off = I.P_off;
        D.compact_base = (long long)compact.size();
        compact.insert(compact.end(), I.compact.begin(), I.compact.end());
    }
    // staging decision and launch shape
    ctx->staged = max_stage <= ctx->smem_optin;
    ctx->smem_bytes = ctx->staged ? std::max<size_t>(max_stage, 16) : 0;
    ctx->grid = ctx->num_sms * (ctx->staged ? 1 : 2);
    // per-mask CTA work ranges over the virtual item list of the enabled parts
    const int G = ctx->grid;
    std::vector<long long> wpre(items.size() + 1, 0);
    for (size_t k = 0; k < items.size(); ++k) wpre[k + 1] = wpre[k] + items[k].len + kItemOverhead;
    std::vector<int> tab(7 * (G + 1), 0);
    std::vector<long long> vpre;
    for (unsigned mask = 1; mask <= 7; ++mask) {
        vpre.assign(1, 0);
        for (int part = 0; part < 3; ++part) {
            if (!(mask & (1u << part))) continue;
            for (int k = ctx->part_first[part]; k < ctx->part_first[part] + ctx->part_items[part]; ++k)
                vpre.push_back(vpre.back() + items[k].len + kItemOverhead);
        }
        const long long total = vpre.back();
        const int nv = (int)vpre.size() - 1;
        int *t = tab.data() + (mask - 1) * (G + 1);
        for (int c = 0; c <= G; ++c) {
            long long target = total * c / G;
            int k = (int)(std::lower_bound(vpre.begin(), vpre.end(), target) - vpre.begin());
            t[c] = std::min(k, nv);
        }
        t[0] = 0;
        t[G] = nv;
    }
    int rc;
    if ((rc = upload_vec(ctx, ctx->items, items))) return rc;
    if ((rc = upload_vec(ctx, ctx->groups, groups))) return rc;
    if ((rc = upload_vec(ctx, ctx->eoff, eoff))) return rc;
    if ((rc = upload_vec(ctx, ctx->poff, poff))) return rc;
    if ((rc = upload_vec(ctx, ctx->ppoff, ppoff))) return rc;
    if ((rc = upload_vec(ctx, ctx->instdev, idev))) return rc;
    if ((rc = upload_vec(ctx, ctx->compact, compact))) return rc;
    if ((rc = upload_vec(ctx, ctx->cta_tab, tab))) return rc;
    ctx->partials.release();
    size_t pb = std::max<size_t>(2 * R * (size_t)std::max(ctx->n_items, 1), 16);
    RT_CUDA(ctx, cudaMalloc(&ctx->partials.p, pb));
    ctx->partials.bytes = pb;
    RT_CUDA(ctx, cudaMemsetAsync(ctx->partials.p, 0, pb, ctx->stream));
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->staged) {
        if (ctx->precision == RTBTE_PREC_FP64)
            RT_CUDA(ctx, cudaFuncSetAttribute(rhs_kernel<double, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)ctx->smem_bytes));
        else
            RT_CUDA(ctx, cudaFuncSetAttribute(rhs_kernel<float, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)ctx->smem_bytes));
    }
    ctx->plan_valid = true;
    return RTBTE_OK;
}

int launch_prep_from_y(rtbte_ctx *ctx, const double *y, cudaStream_t s) {
    RowParams Q = row_params(ctx);
    const int threads = 256;
    const int blocks = (int)std::min<long long>((ctx->n_y + threads - 1) / threads, 8LL * ctx->num_sms);
    if (ctx->precision == RTBTE_PREC_FP64)
        prep_kernel<double><<<blocks, threads, 0, s>>>(Q, y, ctx->n_y);
    else
        prep_kernel<float><<<blocks, threads, 0, s>>>(Q, y, ctx->n_y);
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    return RTBTE_OK;
}

template <class R>
static int launch_core_t(rtbte_ctx *ctx, unsigned parts, const Ctl *ctl, cudaStream_t s) {
    KParams P;
    std::memset(&P, 0, sizeof(P));
    P.items = ctx->items.as<Item>();
    P.groups = ctx->groups.as<Group>();
    P.n_groups = ctx->n_groups;
    P.cta_v = ctx->cta_tab.as<int>() + (parts - 1) * (ctx->grid + 1);
    int v = 0;
    for (int part = 0; part < 3; ++part)
        if (parts & (1u << part)) {
            P.rv[P.nranges] = v;
            P.ri[P.nranges] = ctx->part_first[part];
            P.rlen[P.nranges] = ctx->part_items[part];
            v += ctx->part_items[part];
            P.nranges++;
        }
    P.partials = ctx->partials.p;
    P.popf = ctx->popf.p;
    P.popN = ctx->popN.p;
    P.popP = ctx->popP.p;
    P.ctl = ctl;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ctx->timing) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        RT_CUDA(ctx, cudaStreamIsCapturing(s, &cs));
        if (cs == cudaStreamCaptureStatusNone) {
            for (cudaEvent_t *e : {&e0, &e1}) {
                if (ctx->ev_pool.empty()) {
                    cudaEvent_t ne;
                    RT_CUDA(ctx, cudaEventCreate(&ne));
                    ctx->ev_pool.push_back(ne);
                }
                *e = ctx->ev_pool.back();
                ctx->ev_pool.pop_back();
            }
            RT_CUDA(ctx, cudaEventRecord(e0, s));
        }
    }
    if (ctx->staged) {
        rhs_kernel<R, true, 1><<<ctx->grid, ctx->threads, ctx->smem_bytes, s>>>(P);
    } else {
        rhs_kernel<R, false, 2><<<ctx->grid, ctx->threads, 0, s>>>(P);
    }
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    if (e0) {
        RT_CUDA(ctx, cudaEventRecord(e1, s));
        ctx->ev_pending.push_back({e0, e1});
    }
    return RTBTE_OK;
}

int launch_rhs_core(rtbte_ctx *ctx, unsigned parts, const Ctl *ctl, cudaStream_t s) {
    if (parts == 0 || parts > 7) return fail(ctx, RTBTE_E_INVALID_ARG, "parts must be a non-empty subset of RTBTE_ALL");
    return ctx->precision == RTBTE_PREC_FP64 ? launch_core_t<double>(ctx, parts, ctl, s)
                                             : launch_core_t<float>(ctx, parts, ctl, s);
}

int launch_rows(rtbte_ctx *ctx, unsigned parts, double *out, const double *forcing, cudaStream_t s) {
    RowParams Q = row_params(ctx);
    const int threads = 256;
    const int blocks = (int)std::min<long long>((ctx->n_y + threads - 1) / threads, 8LL * ctx->num_sms);
    if (ctx->precision == RTBTE_PREC_FP64)
        rows_kernel<double><<<blocks, threads, 0, s>>>(Q, parts, out, forcing, ctx->n_y);
    else
        rows_kernel<float><<<blocks, threads, 0, s>>>(Q, parts, out, forcing, ctx->n_y);
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    return RTBTE_OK;
}

}  // namespace rtbte
