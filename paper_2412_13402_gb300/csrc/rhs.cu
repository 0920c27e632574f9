// rhs.cu -- the collision-integral kernels (Eq. e-ph, Eq. ph-ph) and their execution plan.
//
// One persistent launch evaluates the selected parts of the RHS for every instance.  The
// stored channel entries are streamed from HBM exactly once per evaluation (16-byte
// cache-streaming loads, 4 entries per lane), while the populations they gather are
// staged per CTA in shared memory: the instance's electron occupations f plus, for e-ph
// work, the occupations N of one phonon mode, or of one wavevector block of it where the
// whole mode does not fit (the e-ph lists are blocked by mode and block for this reason); for
// ph-e work only f; for ph-ph work the sub-lattice N.  A work item is a piece
// of a single destination segment; groups of long segments give each warp one item of up to
// 512 entries, groups of short ones give each sub-warp of 4, 8 or 16 lanes one item of up to 64,
// 128 or 256 entries.  Lanes accumulate their entries with
// compensated (two-sum) additions in FP32, plain ones in FP64, and add the lanes with a shuffle
// tree; the partial is
// written per item to the item's slot -- the slots of one row's items are consecutive -- and
// the row kernels add a row's partials in slot order (deterministic).  CTAs
// first run a static share of the items (split by estimated cost), then take the rest in
// chunks from a counter; warps may prefetch upcoming items' entries into L2.  FP32 launches
// come in two forms, chosen per parts mask: two register buffers of entries per warp (the next
// item's loads in flight during the current one's arithmetic) at 16 warps per SM, or one buffer
// at 24 warps per SM.
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

// A lane's sum of its (at most 4) vector sums within an item: compensated in FP32; a plain
// addition in FP64, whose rounding over 4 terms is far below the FP64 study's needs and whose
// arithmetic this GPU runs at a low rate (the compensated form cost FP64 mode ~20% of its time).
template <class R> __device__ __forceinline__ void lane_add(R &s, R &c, R x) {
    if constexpr (sizeof(R) == 8) s += x;
    else two_sum(s, c, x);
}

struct KParams {
    const ItemRec *items;
    const Group *groups;
    int n_groups;
    const int *cta_items;  // [grid+1] first item of each CTA's static range (real item indices)
    unsigned mask;         // parts evaluated (groups of other parts are skipped)
    void *partials;
    const void *popf, *popN, *popP;
    const Ctl *ctl;  // per-instance controllers: launches inside an integrator skip finished instances
    const int *act;      // batched integration: active groups in order (-1 ends), else null
    const int *cta_act;  // batched integration: index in act[] of each CTA's first group
    const int4 *tail;  // dynamic chunks {first item, end item, group, 0} after the static ranges
    int n_tail;
    int *tail_ctr;     // [0] next chunk to take, [1] CTAs finished (reset by the last one)
    int pf_dist;       // L2 prefetch distance in items of a warp's sequence (0: off)
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

// Fields of a group that the item loop needs, held in registers.
template <class R> struct GroupView {
    const uint32_t *idx;
    const R *W;
    const R *s0, *s1;  // staged (or global) populations: e-ph f & N of one mode, ph-e f, ph-ph N
    const R *Nglob;    // instance phonon populations (ph-e destinations)
    int part, sb, pb;
    int lg;  // lanes per item = 1 << lg
};

// Entry loads of one item on a sub-warp of 1 << lg lanes: VPL vectors of 4 entries per lane
// (16-byte streaming loads); sl is the lane's index in its sub-warp.
template <class R, int VPL> struct Batch;
template <int VPL> struct Batch<float, VPL> {
    uint4 iv[VPL];
    float4 wv[VPL];
    float Np;  // ph-e destination population, loaded with the entries
    __device__ __forceinline__ void issue(const GroupView<float> &V, const Item &it, int sl, int lg) {
        const int nv = it.len >> 2;
        if (V.part == PART_PHE) Np = V.Nglob[it.dest];
        const uint4 *ip = reinterpret_cast<const uint4 *>(V.idx + it.begin);
        const float4 *wp = reinterpret_cast<const float4 *>(V.W + it.begin);
#pragma unroll
        for (int j = 0; j < VPL; ++j) {
            const int v = sl + (j << lg);
            if (v < nv) {
                iv[j] = __ldcs(ip + v);
                wv[j] = __ldcs(wp + v);
            }
        }
    }
    __device__ __forceinline__ float w(int j, int k) const {
        return k == 0 ? wv[j].x : k == 1 ? wv[j].y : k == 2 ? wv[j].z : wv[j].w;
    }
};
template <int VPL> struct Batch<double, VPL> {
    uint4 iv[VPL];
    double2 wa[VPL], wb[VPL];
    double Np;  // ph-e destination population, loaded with the entries
    __device__ __forceinline__ void issue(const GroupView<double> &V, const Item &it, int sl, int lg) {
        const int nv = it.len >> 2;
        if (V.part == PART_PHE) Np = V.Nglob[it.dest];
        const uint4 *ip = reinterpret_cast<const uint4 *>(V.idx + it.begin);
        const double2 *wp = reinterpret_cast<const double2 *>(V.W + it.begin);
#pragma unroll
        for (int j = 0; j < VPL; ++j) {
            const int v = sl + (j << lg);
            if (v < nv) {
                iv[j] = __ldcs(ip + v);
                wa[j] = __ldcs(wp + 2 * v);
                wb[j] = __ldcs(wp + 2 * v + 1);
            }
        }
    }
    __device__ __forceinline__ double w(int j, int k) const {
        return k == 0 ? wa[j].x : k == 1 ? wa[j].y : k == 2 ? wb[j].x : wb[j].y;
    }
};

__device__ __forceinline__ unsigned comp4(const uint4 &e, int k) {
    return k == 0 ? e.x : k == 1 ? e.y : k == 2 ? e.z : e.w;
}

// Per-lane sum of W*F over one item: each 4-entry vector is summed with an FMA chain and the
// vector sums are added into (acc, cmp) by lane_add; the warp reduction follows in finish_item.
template <class R, int VPL>
__device__ __forceinline__ void compute_item(const GroupView<R> &V, const Item &it, const Batch<R, VPL> &b, int sl,
                                             int lg, R &acc, R &cmp) {
    const int nv = it.len >> 2;
    acc = R(0);
    cmp = R(0);
    if (V.part == PART_EPH) {
        const unsigned smask = (1u << V.sb) - 1u;
        const R fd = V.s0[it.dest];
        if (it.proc == 0) {  // F_em = f(1-f') + N(f-f') = fma(N, f-f', fma(f', -f, f))
#pragma unroll
            for (int j = 0; j < VPL; ++j) {
                if (sl + (j << lg) >= nv) continue;
                R t = R(0);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned e = comp4(b.iv[j], k);
                    const R fs = V.s0[e & smask], N = V.s1[e >> V.sb];
                    const R F = fma(N, fd - fs, fma(fs, -fd, fd));
                    t = fma(b.w(j, k), F, t);
                }
                lane_add(acc, cmp, t);
            }
        } else {  // F_abs = N(f-f') - f'(1-f)
            const R u = R(1) - fd;
#pragma unroll
            for (int j = 0; j < VPL; ++j) {
                if (sl + (j << lg) >= nv) continue;
                R t = R(0);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned e = comp4(b.iv[j], k);
                    const R fs = V.s0[e & smask], N = V.s1[e >> V.sb];
                    const R F = fma(N, fd - fs, -fs * u);
                    t = fma(b.w(j, k), F, t);
                }
                lane_add(acc, cmp, t);
            }
        }
    } else if (V.part == PART_PHE) {  // F_abs(f_d, f_s, N_p) with N_p per item
        const unsigned smask = (1u << V.sb) - 1u;
        const R Np = b.Np;
#pragma unroll
        for (int j = 0; j < VPL; ++j) {
            if (sl + (j << lg) >= nv) continue;
            R t = R(0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned e = comp4(b.iv[j], k);
                const R fd = V.s0[e & smask], fs = V.s0[e >> V.sb];
                const R F = fma(Np, fd - fs, -fs * (R(1) - fd));
                t = fma(b.w(j, k), F, t);
            }
            lane_add(acc, cmp, t);
        }
    } else {
        const unsigned pmask = (1u << V.pb) - 1u;
        const R Na = V.s0[it.dest];
        if (it.proc == 0) {  // G_em = N(N'+N''+1) - N'N''
#pragma unroll
            for (int j = 0; j < VPL; ++j) {
                if (sl + (j << lg) >= nv) continue;
                R t = R(0);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned e = comp4(b.iv[j], k);
                    const R Nb = V.s0[e & pmask], Nc = V.s0[e >> V.pb];
                    const R G = fma(-Nb, Nc, fma(Na, Nb + Nc, Na));
                    t = fma(b.w(j, k), G, t);
                }
                lane_add(acc, cmp, t);
            }
        } else {  // G_abs = N(N''-N') - N'(N''+1)
#pragma unroll
            for (int j = 0; j < VPL; ++j) {
                if (sl + (j << lg) >= nv) continue;
                R t = R(0);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned e = comp4(b.iv[j], k);
                    const R Nb = V.s0[e & pmask], Nc = V.s0[e >> V.pb];
                    const R G = fma(Na, Nc - Nb, -Nb * (Nc + R(1)));
                    t = fma(b.w(j, k), G, t);
                }
                lane_add(acc, cmp, t);
            }
        }
    }
}

__device__ __forceinline__ Item item_from(const int4 &d) {  // decode an ItemRec
    Item it;
    it.begin = ((long long)((unsigned)d.w >> 24) << 32) | (unsigned)d.x;
    it.slot = (unsigned)d.y;
    it.dest = d.z;
    it.len = (unsigned short)(d.w & 0xffff);
    it.proc = (unsigned char)((d.w >> 16) & 0xff);
    return it;
}

// Item descriptors of a warp's strided sequence are fetched 32 at a time (one per lane) and
// broadcast with shuffles.
struct DescStream {
    const int4 *items;
    int k0, end, stride;  // first item of the current block, end of the range, item stride
    int4 cur, nxt;        // this lane's descriptor in the current / next block
    __device__ __forceinline__ int4 fetch(int base, int lane) const {
        const int k = base + lane * stride;
        return k < end ? __ldg(items + k) : make_int4(0, 0, 0, 0);
    }
    __device__ __forceinline__ void init(const ItemRec *it, int a, int b, int st, int lane) {
        items = reinterpret_cast<const int4 *>(it);
        k0 = a;
        end = b;
        stride = st;
        cur = fetch(a, lane);
        nxt = fetch(a + 32 * st, lane);
    }
    __device__ __forceinline__ Item get(int k, int lane) {  // k advances by `stride` per call
        if (k - k0 >= 32 * stride) {
            k0 += 32 * stride;
            cur = nxt;
            nxt = fetch(k0 + 32 * stride, lane);
        }
        const int src = (k - k0) / stride;
        int4 d;
        d.x = __shfl_sync(kFull, cur.x, src);
        d.y = __shfl_sync(kFull, cur.y, src);
        d.z = __shfl_sync(kFull, cur.z, src);
        d.w = __shfl_sync(kFull, cur.w, src);
        return item_from(d);
    }
    // descriptor of item kb + h*stride for this lane (h = its sub-warp), kb warp-uniform and
    // advancing by (items per iteration) * stride per call
    __device__ __forceinline__ Item get_sub(int kb, int h) {
        if (kb - k0 >= 32 * stride) {
            k0 += 32 * stride;
            cur = nxt;
            nxt = fetch(k0 + 32 * stride, threadIdx.x & 31);
        }
        const int off = (kb - k0) / stride + h;
        const bool in_cur = off < 32;
        const int src = in_cur ? off : off - 32;
        int4 d;
        d.x = __shfl_sync(kFull, in_cur ? cur.x : nxt.x, src);
        d.y = __shfl_sync(kFull, in_cur ? cur.y : nxt.y, src);
        d.z = __shfl_sync(kFull, in_cur ? cur.z : nxt.z, src);
        d.w = __shfl_sync(kFull, in_cur ? cur.w : nxt.w, src);
        return item_from(d);
    }
    // descriptor of item k in the current or next block, without advancing (warp-uniform k)
    __device__ __forceinline__ Item peek(int k) const {
        const int off = (k - k0) / stride;
        const bool in_cur = off < 32;
        const int src = in_cur ? off : off - 32;
        int4 d;
        d.x = __shfl_sync(kFull, in_cur ? cur.x : nxt.x, src);
        d.y = __shfl_sync(kFull, in_cur ? cur.y : nxt.y, src);
        d.z = __shfl_sync(kFull, in_cur ? cur.z : nxt.z, src);
        d.w = __shfl_sync(kFull, in_cur ? cur.w : nxt.w, src);
        return item_from(d);
    }
};

// L2 prefetch of item k's entry arrays (one bulk prefetch per array, issued by lane 0), so
// that its streaming loads, issued `dist` items later, find the lines in L2.  Warp-uniform k.
template <class R>
__device__ __forceinline__ void prefetch_item(const GroupView<R> &V, const DescStream &D, int k, int b, int lane) {
    if (k >= b || k - D.k0 >= 64 * D.stride) return;
    const Item it = D.peek(k);
    if (lane == 0 && it.len > 0) {
        const uint32_t *ip = V.idx + it.begin;
        const R *wp = V.W + it.begin;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(ip), "r"((unsigned)it.len * 4u) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(wp), "r"((unsigned)(it.len * sizeof(R)))
                     : "memory");
    }
}

// Item sum: the lane's compensated sum (acc + cmp) is rounded once, then added over the
// sub-warp by a butterfly in a fixed order (every lane ends with the same bits).  The RHS error
// is set by the conversion of the populations to FP32 (about 5e-8 relative on the parity
// models), not by this tree: the compensated tree measured the same to two digits.
template <class R>
__device__ __forceinline__ void finish_item(const KParams &P, unsigned slot, bool valid, R acc, R cmp, int sl, int lg) {
    acc += cmp;
    cmp = R(0);
#pragma unroll
    for (int o = 16; o; o >>= 1)
        if (o < (1 << lg)) acc += __shfl_xor_sync(kFull, acc, o);
    if (sl == 0 && valid) {
        R *out = reinterpret_cast<R *>(P.partials) + 2LL * slot;
        out[0] = acc;
        out[1] = cmp;
    }
}

// Items a, a+st, a+2st, ... < b of one group for one warp.  The warp works on G = 32 >> lg
// items at a time, one per sub-warp of 1 << lg lanes (the group's items are cut to at most
// 16 << lg entries, so groups of short segments pack two or four items to a warp).  WIDE is
// the variant for plans whose groups all use whole-warp items (lg = 5 at compile time).  With
// PIPE, the next items' entry loads are in flight while the current ones are computed (two
// register buffers).
template <class R, bool PIPE, bool WIDE>
__device__ __forceinline__ void run_range(const KParams &P, const GroupView<R> &V, int a, int b, int st, int lane) {
    if (a >= b) return;
    const int lg = WIDE ? 5 : V.lg;
    const int G = 32 >> lg;
    const int h = lane >> lg, sl = lane & ((1 << lg) - 1);
    DescStream D;
    D.init(P.items, a, b, st, lane);
    auto next = [&](int kb) { return WIDE ? D.get(kb, lane) : D.get_sub(kb, h); };
    auto valid = [&](int kb) { return WIDE || kb + h * st < b; };
    const int pf = P.pf_dist;  // iterations ahead whose entries are prefetched into L2 (0: none)
    R acc, cmp;
    if (pf > 0)
        for (int j = 1; j < pf; ++j) prefetch_item(V, D, a + j * G * st, b, lane);
    if (!PIPE) {
        for (int k = a; k < b; k += G * st) {
            const Item it = next(k);
            if (pf > 0) prefetch_item(V, D, k + pf * G * st, b, lane);
            Batch<R, 4> B;
            B.issue(V, it, sl, lg);
            compute_item<R, 4>(V, it, B, sl, lg, acc, cmp);
            finish_item<R>(P, it.slot, valid(k), acc, cmp, sl, lg);
        }
        return;
    }
    Batch<R, 4> A, B;
    int k = a;
    Item ia = next(k);
    A.issue(V, ia, sl, lg);
    for (;;) {
        const bool hb = k + G * st < b;
        Item ib;
        if (hb) {
            ib = next(k + G * st);
            B.issue(V, ib, sl, lg);
        }
        if (pf > 0) prefetch_item(V, D, k + pf * G * st, b, lane);
        compute_item<R, 4>(V, ia, A, sl, lg, acc, cmp);
        finish_item<R>(P, ia.slot, valid(k), acc, cmp, sl, lg);
        if (!hb) break;
        k += G * st;
        const bool ha = k + G * st < b;
        if (ha) {
            ia = next(k + G * st);
            A.issue(V, ia, sl, lg);
        }
        if (pf > 0) prefetch_item(V, D, k + pf * G * st, b, lane);
        compute_item<R, 4>(V, ib, B, sl, lg, acc, cmp);
        finish_item<R>(P, ib.slot, valid(k), acc, cmp, sl, lg);
        if (!ha) break;
        k += G * st;
    }
}

// Point V at group g's populations, staging them in shared memory unless this CTA already
// holds them (`staged` is the group currently in shared memory).  Called by all threads.
template <class R, bool STAGED>
__device__ __forceinline__ void enter_group(const KParams &P, int g, R *sm, int &staged, GroupView<R> &V) {
    const Group &G = P.groups[g];
    V.idx = G.idx;
    V.W = reinterpret_cast<const R *>(G.W);
    V.part = G.part;
    V.sb = G.s_bits;
    V.pb = G.pp_bits;
    V.lg = G.lanes_log2;
    V.Nglob = reinterpret_cast<const R *>(P.popN) + G.N_inst;
    const R *src0 = reinterpret_cast<const R *>(G.part == PART_PP ? P.popP : P.popf) + G.stage0_src;
    const R *src1 = reinterpret_cast<const R *>(P.popN) + G.stage1_src;
    if (STAGED) {
        const int l0 = G.stage0_len, l1 = G.stage1_len;
        if (staged != g) {
            __syncthreads();  // the previous group's readers are done with the buffer
            stage_copy<R>(sm, src0, l0);
            if (l1 > 0) stage_copy<R>(sm + l0, src1, l1);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            __syncthreads();
            staged = g;
        }
        V.s0 = sm;
        V.s1 = sm + l0 - G.stage1_q0;  // indexed by the full q index of the mode
    } else {
        V.s0 = src0;
        V.s1 = src1 - G.stage1_q0;
    }
}

// Persistent collision kernel.  Each CTA first runs its static range of items (cta_items,
// split by estimated cost), then takes dynamic chunks of the remaining items from a shared
// counter until none is left, so that SMs that finish early absorb the tail of the work.
// Items are round-robin over the warps of the CTA; every item writes its own partial, so the
// result does not depend on which CTA ran it.
template <class R, bool STAGED, bool PIPE, bool WIDE, int MINB, int NT>
__global__ void __launch_bounds__(NT, MINB) rhs_kernel(KParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_chunk;
    R *sm = reinterpret_cast<R *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int staged = -1;
    const int ra = P.cta_items[blockIdx.x], rb = P.cta_items[blockIdx.x + 1];
    int g = P.n_groups;  // next group of the static range (with P.act: next index into act[])
    if (ra < rb) {
        if (P.act) {
            g = P.cta_act[blockIdx.x];
        } else {
            int lo = 0, hi = P.n_groups - 1;  // last group with item_begin <= ra
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (P.groups[mid].item_begin <= ra) lo = mid; else hi = mid - 1;
            }
            g = lo;
        }
    }
    bool dynamic = false;
    for (;;) {
        int ug, ua, ub;  // next unit of work: items [ua, ub) of group ug
        if (!dynamic) {
            const int gg = !P.act ? g : (g < P.n_groups ? P.act[g] : -1);
            if (gg < 0 || gg >= P.n_groups || P.groups[gg].item_begin >= rb) {
                dynamic = true;
                if (P.n_tail == 0) break;
                continue;
            }
            ug = gg;
            ++g;
            ua = max(ra, P.groups[ug].item_begin);
            ub = min(rb, P.groups[ug].item_end);
            if (ua >= ub) continue;
        } else {
            __syncthreads();  // every warp is done with the previous unit and with s_chunk
            if (threadIdx.x == 0) s_chunk = atomicAdd(P.tail_ctr, 1);
            __syncthreads();
            const int c = s_chunk;
            if (c >= P.n_tail) break;
            const int4 ch = P.tail[c];
            ug = ch.z;
            ua = ch.x;
            ub = ch.y;
        }
        const Group &G = P.groups[ug];
        if (!(P.mask & (1u << G.part))) continue;
        if (P.ctl && P.ctl[G.inst].done) continue;  // instance already at its t_out
        GroupView<R> V;
        enter_group<R, STAGED>(P, ug, sm, staged, V);
        run_range<R, PIPE, WIDE>(P, V, ua + warp, ub, nwarps, lane);
    }
    if (dynamic && P.n_tail > 0 && threadIdx.x == 0) {  // the last CTA out resets the counters
        __threadfence();
        if (atomicAdd(P.tail_ctr + 1, 1) == (int)gridDim.x - 1) {
            P.tail_ctr[0] = 0;
            P.tail_ctr[1] = 0;
            __threadfence();
        }
    }
}

// Work split over the groups still active (instance not done, part in the mask), recomputed
// on the device before a collision launch inside a batched integration.  One block:
//   - the active groups are listed in order in act[] (terminated by -1);
//   - CTA c gets the active weight [c, c+1) * total / grid: out[c] is its first item, found by
//     interpolating linearly within the active group holding that weight (items of one group
//     carry similar weights; the split affects balance only, never results), and out_act[c]
//     the index in act[] of that group;
//   - out[grid] is the end of the last active group's items.
// A CTA then visits only the active groups act[out_act[c]], ... overlapping its item range,
// so finished instances cost it nothing.
__global__ void split_kernel(const Group *groups, int n_groups, const long long *gw, const Ctl *ctl, unsigned mask,
                             int grid, int *out, int *out_act, int *act, int *memo, int n_inst) {
    __shared__ long long A[1025];   // inclusive prefix of active weight over groups (A[0] = 0)
    __shared__ int Cn[1025];        // active groups before group g
    __shared__ long long wsum[32];
    __shared__ int csum[32];
    __shared__ int s_same;
    const int T = blockDim.x;  // 256 threads, n_groups <= 1024 (checked on the host)
    // the tables of the last split still hold when the same instances are active for the same
    // parts (memo: the done flags and mask it was made for, and a flag the host clears whenever
    // the item weights change)
    if (threadIdx.x == 0) s_same = memo[n_inst + 1] == 1 && memo[n_inst] == (int)mask;
    __syncthreads();
    for (int i = threadIdx.x; i < n_inst; i += T)
        if (memo[i] != ctl[i].done) s_same = 0;
    __syncthreads();
    if (s_same) return;
    const int C = (n_groups + T - 1) / T;
    const int g0 = threadIdx.x * C;
    long long run = 0;
    int nrun = 0;
    for (int g = g0; g < g0 + C && g < n_groups; ++g) {
        const Group &G = groups[g];
        const bool on = (mask & (1u << G.part)) && !ctl[G.inst].done && G.item_end > G.item_begin;
        run += on ? gw[g] : 0;
        nrun += on ? 1 : 0;
        A[g + 1] = run;
        Cn[g + 1] = nrun;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long incl = run;
    int nincl = nrun;
    for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, incl, o);
        const int nv = __shfl_up_sync(0xffffffffu, nincl, o);
        if (lane >= o) {
            incl += v;
            nincl += nv;
        }
    }
    if (lane == 31) {
        wsum[wid] = incl;
        csum[wid] = nincl;
    }
    if (threadIdx.x == 0) {
        A[0] = 0;
        Cn[0] = 0;
    }
    __syncthreads();
    if (wid == 0) {
        long long w = lane < (T >> 5) ? wsum[lane] : 0;
        int nw = lane < (T >> 5) ? csum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long v = __shfl_up_sync(0xffffffffu, w, o);
            const int nv = __shfl_up_sync(0xffffffffu, nw, o);
            if (lane >= o) {
                w += v;
                nw += nv;
            }
        }
        if (lane < (T >> 5)) {
            wsum[lane] = w;
            csum[lane] = nw;
        }
    }
    __syncthreads();
    const long long before = incl - run + (wid > 0 ? wsum[wid - 1] : 0);
    const int nbefore = nincl - nrun + (wid > 0 ? csum[wid - 1] : 0);
    for (int g = g0; g < g0 + C && g < n_groups; ++g) {
        A[g + 1] += before;
        Cn[g + 1] += nbefore;
    }
    __syncthreads();
    const long long total = A[n_groups];
    const int n_act = Cn[n_groups];
    for (int g = threadIdx.x; g < n_groups; g += T)  // compact list of the active groups
        if (Cn[g + 1] > Cn[g]) act[Cn[g]] = g;
    if (threadIdx.x == 0) act[n_act] = -1;
    for (int c = threadIdx.x; c <= grid; c += T) {
        if (total == 0) {
            out[c] = 0;
            if (c < grid) out_act[c] = 0;
            continue;
        }
        if (c == grid) {  // end of the last active group's items
            int last = n_groups - 1;
            while (last > 0 && Cn[last + 1] == Cn[last]) --last;
            out[c] = groups[last].item_end;
            continue;
        }
        const long long t = total * c / grid;
        int lo = 0, hi = n_groups - 1;  // group g with A[g] <= t < A[g+1]
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (A[mid] <= t) lo = mid; else hi = mid - 1;
        }
        while (lo < n_groups - 1 && A[lo + 1] == A[lo]) ++lo;  // skip inactive groups
        const Group &G = groups[lo];
        const long long wg = A[lo + 1] - A[lo];
        const long long ni = G.item_end - G.item_begin;
        out[c] = G.item_begin + (int)((t - A[lo]) * ni / (wg > 0 ? wg : 1));
        out_act[c] = Cn[lo];
    }
    for (int i = threadIdx.x; i < n_inst; i += T) memo[i] = ctl[i].done;
    if (threadIdx.x == 0) {
        memo[n_inst] = (int)mask;
        memo[n_inst + 1] = 1;
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
    Q.rowoff = ctx->rowoff.as<int>();
    Q.rowmid = ctx->rowmid.as<int>();
    Q.compact = ctx->compact.as<int>();
    Q.partials = ctx->partials.p;
    Q.popf = ctx->popf.p;
    Q.popN = ctx->popN.p;
    Q.popP = ctx->popP.p;
    return Q;
}

// Per-mask work split of the persistent grid.  Item weight = (entries + w) x the part's
// calibrated cost per entry, with each mask's own w and costs.  The first share sf of a mask's
// weight is split into equal-weight contiguous CTA ranges (table [mask][grid+1] of real item
// indices); the rest is
// cut into dynamic chunks of decreasing weight (half the remaining weight per grid, at least
// 1/40 of a CTA's share, never across a group boundary), taken by CTAs in order at run time.
int split_tables(rtbte_ctx *ctx) {
    const int G = ctx->grid;
    const std::vector<unsigned short> &len = ctx->item_len_h;
    const int n = (int)len.size();
    // weight of item k under mask m's parameters: (entries + w) x the part's cost per entry
    auto weight = [&](const LaunchTuning &L, int part, int k) {
        const long long sc = (long long)(64.0 * L.ps[part] + 0.5);  // cost per entry-equivalent
        return sc * (len[k] + L.w);
    };
    std::vector<int> item_group(n, 0);
    for (size_t g = 0; g < ctx->group_begin_h.size(); ++g) {
        const int e = g + 1 < ctx->group_begin_h.size() ? ctx->group_begin_h[g + 1] : n;
        for (int k = ctx->group_begin_h[g]; k < e; ++k) item_group[k] = (int)g;
    }
    std::vector<int> tab(7LL * (G + 1), 0);
    std::vector<int4> tail;
    std::vector<long long> apre;  // prefix of the enabled parts' weights, item order
    std::vector<int> aidx;
    for (unsigned mask = 1; mask <= 7; ++mask) {
        const LaunchTuning &L = ctx->lt[mask];
        apre.assign(1, 0);
        aidx.clear();
        for (int part = 0; part < 3; ++part) {
            if (!(mask & (1u << part))) continue;
            for (int k = ctx->part_first[part]; k < ctx->part_first[part] + ctx->part_items[part]; ++k) {
                apre.push_back(apre.back() + weight(L, part, k));
                aidx.push_back(k);
            }
        }
        const long long total = apre.back();
        const int na = (int)aidx.size();
        const long long split = L.sf >= 1.0 ? total : (long long)(L.sf * (double)total);
        const int js = (int)(std::lower_bound(apre.begin(), apre.end(), split) - apre.begin());  // first tail item
        int *t = tab.data() + (long long)(mask - 1) * (G + 1);
        for (int c = 0; c <= G; ++c) {
            if (na == 0) {
                t[c] = 0;
                continue;
            }
            if (c == G) {
                t[c] = js >= na ? n : aidx[js];
                continue;
            }
            const long long target = split * c / G;
            const int j = (int)(std::lower_bound(apre.begin(), apre.end(), target) - apre.begin());
            t[c] = c == 0 ? 0 : (j >= na ? n : (j >= js ? aidx[js] : aidx[j]));
        }
        const long long wmin = std::max<long long>(1, total / (40LL * G));
        for (int j = js; j < na;) {
            const long long remaining = total - apre[j];
            const long long want = std::max(wmin, remaining / (2LL * G));
            const int g = item_group[aidx[j]];
            int j2 = j + 1;
            while (j2 < na && item_group[aidx[j2]] == g && aidx[j2] == aidx[j2 - 1] + 1 && apre[j2] - apre[j] < want)
                ++j2;
            tail.push_back(make_int4(aidx[j], aidx[j2 - 1] + 1, g, 0));
            j = j2;
        }
        ctx->tail_off[mask] = (int)tail.size();
    }
    // per-group weights for the device re-split of batched integrations (full-RHS parameters)
    std::vector<long long> wpre(n + 1, 0);
    for (int part = 0; part < 3; ++part)
        for (int k = ctx->part_first[part]; k < ctx->part_first[part] + ctx->part_items[part]; ++k)
            wpre[k + 1] = weight(ctx->lt[7], part, k);
    for (int k = 0; k < n; ++k) wpre[k + 1] += wpre[k];
    std::vector<long long> gwt(ctx->group_begin_h.size());  // weight of each group's items
    for (size_t g = 0; g < gwt.size(); ++g) {
        const int e = g + 1 < ctx->group_begin_h.size() ? ctx->group_begin_h[g + 1] : n;
        gwt[g] = wpre[e] - wpre[ctx->group_begin_h[g]];
    }
    int rc;
    if ((rc = upload_vec(ctx, ctx->gwt, gwt))) return rc;
    // the device re-split's memo no longer matches the weights: clear its valid flag
    const size_t valid_at = 2 * (size_t)ctx->grid + 1 + ctx->n_groups + 1 + ctx->inst.size() + 1;
    if (ctx->dyn_tab.p && (valid_at + 1) * sizeof(int) <= ctx->dyn_tab.bytes)
        RT_CUDA(ctx, cudaMemsetAsync(ctx->dyn_tab.as<int>() + valid_at, 0, sizeof(int), ctx->stream));
    if (tail.empty()) tail.push_back(make_int4(0, 0, 0, 0));
    if ((rc = upload_vec(ctx, ctx->tail_tab, tail))) return rc;
    return upload_vec(ctx, ctx->cta_tab, tab);
}

// Build the work items, staging groups, per-row partial slots and per-CTA work ranges.
int make_plan(rtbte_ctx *ctx) {
    const size_t R = ctx->real_size;
    std::vector<ItemRec> items;
    std::vector<Group> groups;
    std::vector<int> eoff, poff, ppoff;  // item offsets per row (host only: they order the slots)
    std::vector<long long> eoff_base(ctx->inst.size()), poff_base(ctx->inst.size()), ppoff_base(ctx->inst.size());
    std::vector<InstDev> idev(ctx->inst.size());
    bool begin_overflow = false;
    int cut = 512;  // entries per item at most (16 << the current group's lanes_log2)
    // lanes per item of a group: from the mean padded length of its non-empty segments [s0, s1),
    // counted over every row (also those outside a row slice, so that a sliced context cuts
    // its items as a full one does), so that a sub-warp's item holds about one segment
    auto lanes_log2 = [](const std::vector<long long> &plen, long long s0, long long s1) {
        long long tot = 0, n = 0;
        for (long long s = s0; s < s1; ++s)
            if (plen[s] > 0) {
                tot += plen[s];
                ++n;
            }
        const double mean = n ? (double)tot / (double)n : 0.0;
        return mean <= 64.0 ? 2 : mean <= 128.0 ? 3 : mean <= 256.0 ? 4 : 5;
    };
    auto add_seg = [&](long long b, long long e, int dest, int proc) {
        for (long long x = b; x < e; x += cut) {
            ItemRec it;
            begin_overflow = begin_overflow || x >= (1LL << 40);
            it.begin_lo = (unsigned)(x & 0xffffffffLL);
            it.begin_hi = (unsigned char)((x >> 32) & 0xff);
            it.slot = 0;  // set once every item exists
            it.dest = dest;
            it.len = (unsigned short)std::min<long long>(cut, e - x);
            it.proc = (unsigned char)proc;
            items.push_back(it);
        }
    };
    size_t max_stage = 0;
    // e-ph groups (instance, mode)
    for (size_t i = 0; i < ctx->inst.size(); ++i) {
        InstHost &I = ctx->inst[i];
        eoff_base[i] = (long long)eoff.size();
        const int nqb = std::max(I.eph_nqb, 1);
        const int qblk = I.eph_qblk > 0 ? I.eph_qblk : I.N_q_pad;
        for (int blk = 0; blk < I.d.nmodes * nqb; ++blk) {  // (mode, q-block)
            const int nu = blk / nqb, qb = blk % nqb;
            const int q_lo = qb * qblk, q_len = std::min(qblk, I.N_q_pad - q_lo);
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
            G.stage1_len = q_len;
            G.stage1_src = I.N_off + (long long)nu * I.N_q_pad + q_lo;
            G.stage1_q0 = q_lo;
            G.lanes_log2 = lanes_log2(I.eph_plen, 2LL * blk * I.d.n_c, 2LL * (blk + 1) * I.d.n_c);
            cut = 16 << G.lanes_log2;
            G.f_inst = I.f_off;
            G.N_inst = I.N_off;
            G.P_inst = I.P_off;
            for (int d = 0; d < I.d.n_c; ++d) {
                eoff.push_back((int)items.size());
                long long g = ((long long)blk * I.d.n_c + d) * 2;
                
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
        poff_base[i] = (long long)poff.size();
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
        G.lanes_log2 = lanes_log2(I.phe_plen, 0, I.n_ph);
        cut = 16 << G.lanes_log2;
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
        ppoff_base[i] = (long long)ppoff.size();
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
        G.lanes_log2 = lanes_log2(I.pp_plen, 0, 2 * I.M);
        cut = 16 << G.lanes_log2;
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
    if (begin_overflow) return fail(ctx, RTBTE_E_UNSUPPORTED, "channel list longer than 2^40 entries");
    // partial slots, row-major: every row's items get consecutive slots in the order the row
    // adds them (an electron row: its (mode, q-block) blocks in turn, emission then absorption
    // items of each; a phonon row: its ph-e items, then its ph-ph items if it is a sub-lattice
    // phonon), so a row kernel reads one offset pair and one contiguous run of partials
    std::vector<int> rowoff(ctx->n_y + 1, 0), rowmid(std::max<long long>(ctx->n_y, 1), 0);
    {
        long long next = 0;
        auto take = [&](int i0, int i1) {
            for (int k = i0; k < i1; ++k) items[k].slot = (unsigned)next++;
        };
        for (size_t i = 0; i < ctx->inst.size(); ++i) {
            const InstHost &I = ctx->inst[i];
            const int nc = I.d.n_c, nblk = I.d.nmodes * std::max(I.eph_nqb, 1);
            for (int d = 0; d < nc; ++d) {
                const long long c = I.y_off + d;
                rowoff[c] = (int)next;
                for (int blk = 0; blk < nblk; ++blk) {
                    const long long o = eoff_base[i] + (long long)blk * (nc + 1) + d;
                    take(eoff[o], eoff[o + 1]);
                }
                rowmid[c] = (int)next;
            }
            for (long long p = 0; p < I.n_ph; ++p) {
                const long long c = I.y_off + nc + p;
                rowoff[c] = (int)next;
                take(poff[poff_base[i] + p], poff[poff_base[i] + p + 1]);
                rowmid[c] = (int)next;
                const int a = I.M > 0 ? I.compact[p] : -1;
                if (a >= 0) take(ppoff[ppoff_base[i] + a], ppoff[ppoff_base[i] + a + 1]);
            }
        }
        rowoff[ctx->n_y] = (int)next;
        if (next != (long long)items.size()) return fail(ctx, RTBTE_E_UNSUPPORTED, "work items not covered by rows");
    }
    ctx->n_items = (int)items.size();
    ctx->n_groups = (int)groups.size();
    ctx->wide = std::all_of(groups.begin(), groups.end(), [](const Group &G) { return G.lanes_log2 == 5; });
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
    // staging decision and launch shape: 16 warps per SM, as 1, 2 or 4 CTAs -- several CTAs
    // per SM when their staging fits, so one CTA's group change (barrier + staging copy)
    // overlaps the others' streaming
    ctx->staged = max_stage + 64 <= ctx->smem_optin;  // 64 B left for the kernel's static shared memory
    ctx->smem_bytes = ctx->staged ? std::max<size_t>(max_stage, 16) : 0;
    // Two forms of the FP32 kernel: two register buffers of entries per warp at 16 warps per SM
    // (128 registers), or one buffer at 24 warps per SM (80 registers), which hides the gather and
    // arithmetic latency better on the e-ph part.  Both must fit the chosen CTAs per SM.
    int per_sm = 1;
    const bool fp64 = ctx->precision == RTBTE_PREC_FP64;
    if (ctx->staged) {
        std::vector<std::pair<const void *, int>> kfns;  // (kernel, threads per SM)
        if (fp64) {
            kfns.push_back({ctx->wide ? (const void *)rhs_kernel<double, true, false, true, 1, kRhsThreads>
                                      : (const void *)rhs_kernel<double, true, false, false, 1, kRhsThreads>,
                            kRhsThreads});
        } else {
            kfns.push_back({ctx->wide ? (const void *)rhs_kernel<float, true, true, true, 1, kRhsThreads>
                                      : (const void *)rhs_kernel<float, true, true, false, 1, kRhsThreads>,
                            kRhsThreads});
            kfns.push_back({ctx->wide ? (const void *)rhs_kernel<float, true, false, true, 1, kRhsThreadsDeep>
                                      : (const void *)rhs_kernel<float, true, false, false, 1, kRhsThreadsDeep>,
                            kRhsThreadsDeep});
        }
        for (auto &kf : kfns) {
            RT_CUDA(ctx, allow_max_dynamic_smem(kf.first));
            RT_CUDA(ctx, cudaFuncSetAttribute(kf.first, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        }
        for (int k : {4, 2}) {
            bool fits = true;
            for (auto &kf : kfns) {
                int nb = 0;
                RT_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kf.first, kf.second / k, ctx->smem_bytes));
                fits = fits && nb >= k;
            }
            if (fits) {
                per_sm = k;
                break;
            }
        }
    }
    ctx->per_sm = per_sm;
    for (unsigned m = 0; m < 8; ++m)  // default: the 768-thread form where e-ph work is in the launch
        if (!(ctx->lt_tuned & (1u << m))) ctx->lt[m].deep = !fp64 && (m & (1u << PART_EPH));
    ctx->grid = ctx->num_sms * (ctx->staged ? per_sm : 2);
    ctx->item_len_h.resize(items.size());
    for (size_t k = 0; k < items.size(); ++k) ctx->item_len_h[k] = items[k].len;
    ctx->group_begin_h.resize(groups.size());
    for (size_t g = 0; g < groups.size(); ++g) ctx->group_begin_h[g] = groups[g].item_begin;
    int rc;
    if (!ctx->tail_ctr.p) {
        RT_CUDA(ctx, cudaMalloc(&ctx->tail_ctr.p, 16));
        ctx->tail_ctr.bytes = 16;
        RT_CUDA(ctx, cudaMemsetAsync(ctx->tail_ctr.p, 0, 16, ctx->stream));
    }
    if ((rc = upload_vec(ctx, ctx->items, items))) return rc;
    if ((rc = upload_vec(ctx, ctx->groups, groups))) return rc;
    if ((rc = upload_vec(ctx, ctx->rowoff, rowoff))) return rc;
    if ((rc = upload_vec(ctx, ctx->rowmid, rowmid))) return rc;
    if ((rc = upload_vec(ctx, ctx->instdev, idev))) return rc;
    if ((rc = upload_vec(ctx, ctx->compact, compact))) return rc;
    if (ctx->n_y >= (long long)INT32_MAX) return fail(ctx, RTBTE_E_UNSUPPORTED, "state vector too long");
    if (ctx->inst.size() > (size_t)kMaxBatch) return fail(ctx, RTBTE_E_UNSUPPORTED, "more than 1024 instances");
    long long nrb = 0;  // row blocks of 256 rows of one instance (batched stage kernels)
    if (ctx->inst.size() > 1)
        for (const InstHost &I : ctx->inst) nrb += (I.d.n_c + I.n_ph + 255) / 256;
    ctx->n_rblk = (int)nrb;
    ctx->dyn_tab.release();  // reallocated below for this plan's sizes
    if ((rc = split_tables(ctx))) return rc;
    if (ctx->n_groups > 1024) return fail(ctx, RTBTE_E_UNSUPPORTED, "more than 1024 staging groups");
    // device re-split tables: [grid+1] item bounds, [grid] act indices, [n_groups+1] active groups,
    // then the memo of the last split: [n_inst] done flags it saw, its parts mask, a valid flag
    ctx->dyn_tab.release();
    ctx->dyn_tab.bytes = sizeof(int) * (2 * ctx->grid + 1 + ctx->n_groups + 1 + ctx->inst.size() + 2);
    RT_CUDA(ctx, cudaMalloc(&ctx->dyn_tab.p, ctx->dyn_tab.bytes));
    RT_CUDA(ctx, cudaMemsetAsync(ctx->dyn_tab.p, 0, ctx->dyn_tab.bytes, ctx->stream));
    ctx->partials.release();
    size_t pb = std::max<size_t>(2 * R * (size_t)std::max(ctx->n_items, 1), 16);
    RT_CUDA(ctx, cudaMalloc(&ctx->partials.p, pb));
    ctx->partials.bytes = pb;
    RT_CUDA(ctx, cudaMemsetAsync(ctx->partials.p, 0, pb, ctx->stream));
    RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if ((rc = init_stage_grid(ctx))) return rc;
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
    P.items = ctx->items.as<ItemRec>();
    P.groups = ctx->groups.as<Group>();
    P.n_groups = ctx->n_groups;
    P.mask = parts;
    P.pf_dist = ctx->lt[parts].pf;
    if (ctl && ctx->inst.size() > 1) {  // batched integration: balance over the active instances
        int *dt = ctx->dyn_tab.as<int>();  // [grid+1] item bounds, [grid] act indices, [n_groups+1] act, memo
        split_kernel<<<1, 256, 0, s>>>(ctx->groups.as<Group>(), ctx->n_groups, ctx->gwt.as<long long>(), ctl, parts,
                                       ctx->grid, dt, dt + ctx->grid + 1, dt + 2 * ctx->grid + 1,
                                       dt + 2 * ctx->grid + 1 + ctx->n_groups + 1, (int)ctx->inst.size());
        RT_CUDA(ctx, cudaGetLastError());
        ctx->launches++;
        P.cta_items = dt;
        P.cta_act = dt + ctx->grid + 1;
        P.act = dt + 2 * ctx->grid + 1;
    } else {
        P.cta_items = ctx->cta_tab.as<int>() + (long long)(parts - 1) * (ctx->grid + 1);
        P.tail = ctx->tail_tab.as<int4>() + ctx->tail_off[parts - 1];
        P.n_tail = ctx->tail_off[parts] - ctx->tail_off[parts - 1];
        P.tail_ctr = ctx->tail_ctr.as<int>();
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
    if (!ctx->staged) {
        rhs_kernel<R, false, false, false, 2, kRhsThreads><<<ctx->grid, kRhsThreads, 0, s>>>(P);
    } else if constexpr (sizeof(R) == 4) {
        if (ctx->lt[parts].deep) {
            const int nt = kRhsThreadsDeep / ctx->per_sm;
            if (ctx->wide)
                rhs_kernel<R, true, false, true, 1, kRhsThreadsDeep><<<ctx->grid, nt, ctx->smem_bytes, s>>>(P);
            else
                rhs_kernel<R, true, false, false, 1, kRhsThreadsDeep><<<ctx->grid, nt, ctx->smem_bytes, s>>>(P);
        } else {
            const int nt = kRhsThreads / ctx->per_sm;
            if (ctx->wide)
                rhs_kernel<R, true, true, true, 1, kRhsThreads><<<ctx->grid, nt, ctx->smem_bytes, s>>>(P);
            else
                rhs_kernel<R, true, true, false, 1, kRhsThreads><<<ctx->grid, nt, ctx->smem_bytes, s>>>(P);
        }
    } else {
        const int nt = kRhsThreads / ctx->per_sm;
        if (ctx->wide)
            rhs_kernel<R, true, false, true, 1, kRhsThreads><<<ctx->grid, nt, ctx->smem_bytes, s>>>(P);
        else
            rhs_kernel<R, true, false, false, 1, kRhsThreads><<<ctx->grid, nt, ctx->smem_bytes, s>>>(P);
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

namespace {

// Time `reps` collision launches for `parts` after one untimed launch.
int time_launches(rtbte_ctx *ctx, unsigned parts, cudaEvent_t e0, cudaEvent_t e1, int reps, float *ms) {
    int rc;
    if ((rc = launch_rhs_core(ctx, parts, nullptr, ctx->stream))) return rc;
    RT_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
    for (int r = 0; r < reps; ++r)
        if ((rc = launch_rhs_core(ctx, parts, nullptr, ctx->stream))) return rc;
    RT_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    RT_CUDA(ctx, cudaEventSynchronize(e1));
    RT_CUDA(ctx, cudaEventElapsedTime(ms, e0, e1));
    return RTBTE_OK;
}

// Tuning of mask `parts`'s work split for its current kernel form: per-item weight, per-part
// entry costs, L2 prefetch distance and static share, each timed over 3 launches and the
// fastest kept.
int tune_split(rtbte_ctx *ctx, unsigned parts, cudaEvent_t e0, cudaEvent_t e1) {
    static const int cand[] = {32, 96, 192, 320, 512, 800, 1280, 2048};
    LaunchTuning &L = ctx->lt[parts];
    int best = L.w, rc = RTBTE_OK;
    float best_ms = 1e30f;
    for (int w : cand) {
        float ms = 0.f;
        L.w = w;
        if ((rc = split_tables(ctx)) || (rc = time_launches(ctx, parts, e0, e1, 3, &ms))) return rc;
        if (ms < best_ms) {
            best_ms = ms;
            best = w;
        }
    }
    L.w = best;
    if ((rc = split_tables(ctx))) return rc;
    // calibrate the relative cost of an entry in each part from single-part launches (run with
    // this mask's parameters), keep it if this mask's launch gets faster
    const double scale0[3] = {L.ps[0], L.ps[1], L.ps[2]};
    double t[3] = {0, 0, 0}, wsum[3] = {0, 0, 0};
    int used = 0;
    for (int part = 0; part < 3; ++part) {
        if (!(parts & (1u << part)) || ctx->part_items[part] == 0 || (parts == (1u << part))) continue;
        for (int k = ctx->part_first[part]; k < ctx->part_first[part] + ctx->part_items[part]; ++k)
            wsum[part] += ctx->item_len_h[k] + best;
        const unsigned pm = 1u << part;
        const LaunchTuning keep = ctx->lt[pm];
        ctx->lt[pm] = L;
        float ms = 0.f;
        rc = split_tables(ctx);
        if (!rc) rc = time_launches(ctx, pm, e0, e1, 3, &ms);
        ctx->lt[pm] = keep;
        if (rc) return rc;
        t[part] = ms;
        used |= pm;
    }
    if (used) {
        double ref = 0.0;
        int nref = 0;
        for (int part = 0; part < 3; ++part)
            if (used & (1u << part)) {
                ref += t[part] / wsum[part];
                ++nref;
            }
        ref /= nref;
        for (int part = 0; part < 3; ++part)
            if (used & (1u << part)) L.ps[part] = (t[part] / wsum[part]) / ref;
        float ms = 0.f;
        if ((rc = split_tables(ctx)) || (rc = time_launches(ctx, parts, e0, e1, 3, &ms))) return rc;
        if (ms > best_ms) {  // calibration did not help: back to the previous costs
            for (int part = 0; part < 3; ++part) L.ps[part] = scale0[part];
            if ((rc = split_tables(ctx))) return rc;
        }
    }
    // L2 prefetch distance, then the share of the work split statically (the rest is taken
    // dynamically by CTAs that finish early)
    static const int dists[] = {0, 2, 3, 4, 6, 8};
    int best_d = L.pf;
    float best_d_ms = 1e30f;
    for (int d : dists) {
        L.pf = d;
        float ms = 0.f;
        if ((rc = time_launches(ctx, parts, e0, e1, 3, &ms))) return rc;
        if (ms < best_d_ms) {
            best_d_ms = ms;
            best_d = d;
        }
    }
    L.pf = best_d;
    static const double fracs[] = {1.0, 0.9, 0.8, 0.7, 0.6};
    double best_f = 1.0;
    float best_f_ms = 1e30f;
    for (double f : fracs) {
        L.sf = f;
        float ms = 0.f;
        if ((rc = split_tables(ctx)) || (rc = time_launches(ctx, parts, e0, e1, 3, &ms))) return rc;
        if (ms < best_f_ms) {
            best_f_ms = ms;
            best_f = f;
        }
    }
    L.sf = best_f;
    return split_tables(ctx);
}

}  // namespace

// Autotuner of the collision launch of one parts mask.  FP32 has two kernel forms (two entry
// buffers per warp at 16 warps per SM, or one buffer at 24): the work split is tuned for each
// form from the same starting point, the two tuned launches are timed over 10 launches each
// (they often differ by ~2%, less than the spread of 3-launch timings) and the faster is kept.
// The result belongs to this mask; masks never tuned themselves take its work split (not its
// form) as their own.
int autotune(rtbte_ctx *ctx, unsigned parts, int *chosen) {
    cudaEvent_t e0, e1;
    RT_CUDA(ctx, cudaEventCreate(&e0));
    RT_CUDA(ctx, cudaEventCreate(&e1));
    const bool two_forms = ctx->staged && ctx->precision != RTBTE_PREC_FP64;
    const LaunchTuning start = ctx->lt[parts];
    LaunchTuning res[2] = {start, start};
    float ms10[2] = {0.f, 0.f};
    int rc = RTBTE_OK, nf = two_forms ? 2 : 1;
    for (int f = 0; f < nf && !rc; ++f) {
        ctx->lt[parts] = start;
        if (two_forms) ctx->lt[parts].deep = f == 1;
        if ((rc = tune_split(ctx, parts, e0, e1))) break;
        if (two_forms && (rc = time_launches(ctx, parts, e0, e1, 10, &ms10[f]))) break;
        res[f] = ctx->lt[parts];
    }
    const int pick = (!rc && two_forms && ms10[1] < ms10[0]) ? 1 : 0;
    ctx->lt[parts] = rc ? start : res[pick];
    if (!rc) {
        ctx->lt_tuned |= 1u << parts;
        for (unsigned m = 1; m <= 7; ++m) {
            if (m == parts || (ctx->lt_tuned & (1u << m))) continue;
            const bool deep = ctx->lt[m].deep;
            ctx->lt[m] = ctx->lt[parts];
            ctx->lt[m].deep = deep;
        }
    }
    const int rc2 = split_tables(ctx);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (rc2) return rc2;
    if (chosen) *chosen = ctx->lt[parts].w;
    return RTBTE_OK;
}

// Linearised ph-ph rates: one warp per sub-lattice destination a of one instance,
//   Gamma_a = -dI^{ph-ph}_a/dN_a = sum_em W (N' + N'' + 1) + sum_abs W (N'' - N')
// (Eq. ph-ph with G_em, G_abs differentiated in the destination population; W as stored,
// pair and absorption factors included), from the compute-precision sub-lattice copy popP,
// summed in FP64 per lane then a fixed butterfly; written to rates[y_off + n_c + full(a)].
template <class R>
__global__ void pp_rates_kernel(const uint32_t *idx, const R *W, const long long *off, const R *P, const int *pp_full,
                                int pp_bits, long long M, long long row0, double *rates) {
    const int lane = threadIdx.x & 31;
    const unsigned pmask = (1u << pp_bits) - 1u;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long a = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; a < M; a += nw) {
        double acc = 0.0;
        for (int proc = 0; proc < 2; ++proc)
            for (long long e = off[2 * a + proc] + lane; e < off[2 * a + proc + 1]; e += 32) {
                const uint32_t x = idx[e];
                const double Nb = (double)P[x & pmask], Nc = (double)P[x >> pp_bits];
                acc += (double)W[e] * (proc == 0 ? Nb + Nc + 1.0 : Nc - Nb);
            }
#pragma unroll
        for (int m = 16; m; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
        if (lane == 0) rates[row0 + pp_full[a]] = acc;
    }
}

int launch_pp_rates(rtbte_ctx *ctx, int inst, double *rates, cudaStream_t s) {
    InstHost &I = ctx->inst[inst];
    if (I.M == 0) return RTBTE_OK;
    if (!I.pp_off_dev.p) {
        RT_CUDA(ctx, cudaMalloc(&I.pp_off_dev.p, sizeof(long long) * I.pp_off.size()));
        I.pp_off_dev.bytes = sizeof(long long) * I.pp_off.size();
        RT_CUDA(ctx, cudaMemcpyAsync(I.pp_off_dev.p, I.pp_off.data(), I.pp_off_dev.bytes, cudaMemcpyHostToDevice, s));
    }
    const int blocks = (int)std::min<long long>((I.M + 7) / 8, 8LL * ctx->num_sms);
    if (ctx->precision == RTBTE_PREC_FP64)
        pp_rates_kernel<double><<<blocks, 256, 0, s>>>(I.pp_idx.as<uint32_t>(), I.pp_W.as<double>(),
                                                       I.pp_off_dev.as<long long>(),
                                                       ctx->popP.as<double>() + I.P_off, I.t_ppfull.as<int>(),
                                                       I.pp_bits, I.M, I.y_off + I.d.n_c, rates);
    else
        pp_rates_kernel<float><<<blocks, 256, 0, s>>>(I.pp_idx.as<uint32_t>(), I.pp_W.as<float>(),
                                                      I.pp_off_dev.as<long long>(), ctx->popP.as<float>() + I.P_off,
                                                      I.t_ppfull.as<int>(), I.pp_bits, I.M, I.y_off + I.d.n_c, rates);
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    return RTBTE_OK;
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
