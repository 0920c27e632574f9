// rows.cuh -- per-row device helpers shared by the RHS and integrator kernels.
//
// A "row" is one component of the state vector y = [f; N] (Eq. state_vec).  Its RHS value
// is minus the sum of the compensated partial sums of its work items (the collision
// integrals of Eq. e-ph and Eq. ph-ph carry an overall minus sign), accumulated in FP64 in
// item order, so a row's value does not depend on how items were scheduled.
#pragma once

#include "internal.cuh"

namespace rtbte {

struct RowParams {
    const InstDev *inst;
    int n_inst;
    const int *rowoff;               // [n_y+1] first partial slot of each state row
    const int *rowmid;               // [n_y] phonon rows: first ph-ph slot (ph-e slots before it)
    const int *compact;              // sub-lattice index of each phonon or -1
    const void *partials;            // (hi, lo) per item, compute precision
    void *popf, *popN, *popP;        // population copies, compute precision
};

__device__ __forceinline__ int find_inst(const RowParams &Q, long long comp) {
    int lo = 0, hi = Q.n_inst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (Q.inst[mid].y_off <= comp) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Accumulator of item partials (hi, lo) in item order.  FP64 partials add in FP64.  FP32
// partials add as an FP32 head/tail pair (two-sum on the heads, tails summed) and are widened
// once at the end: about 48 significant bits, far below the partials' own rounding, with no
// FP64 arithmetic per item (FP64 throughput is low on this GPU).
template <class R> struct RowAcc {
    double acc = 0.0;
    __device__ __forceinline__ void add(R hi, R lo) { acc += (double)hi + (double)lo; }
    __device__ __forceinline__ double value() const { return acc; }
};
template <> struct RowAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float hi, float lo) {
        const float t = s + hi;
        const float bp = t - s;
        c += ((s - (t - bp)) + (hi - bp)) + lo;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <class R>
__device__ __forceinline__ void item_sum(const RowParams &Q, int i0, int i1, RowAcc<R> &A) {
    const R *P = reinterpret_cast<const R *>(Q.partials);
    for (int it = i0; it < i1; ++it) A.add(P[2 * it], P[2 * it + 1]);
}

// RHS value of row `local` of instance I for the selected parts.  The row's partials sit in
// consecutive slots: an electron row's e-ph items in (mode, q-block) order, a phonon row's ph-e
// items then its ph-ph items (sub-lattice phonons only).
template <class R>
__device__ __forceinline__ double row_value(const RowParams &Q, const InstDev &I, long long local, unsigned parts) {
    const long long c = I.y_off + local;
    const int s0 = Q.rowoff[c], s1 = Q.rowmid[c], s2 = Q.rowoff[c + 1];
    RowAcc<R> A;
    if (local < I.n_c) {
        if (!(parts & RTBTE_EPH)) return 0.0;
        item_sum<R>(Q, s0, s2, A);
        return -A.value();
    }
    if (parts & RTBTE_PHE) item_sum<R>(Q, s0, s1, A);
    if (parts & RTBTE_PHPH) item_sum<R>(Q, s1, s2, A);
    return -A.value();
}

// Store component value v of row `local` into the population copies read by the RHS.
template <class R>
__device__ __forceinline__ void write_pops(const RowParams &Q, const InstDev &I, long long local, R v) {
    if (local < I.n_c) {
        reinterpret_cast<R *>(Q.popf)[I.f_off + local] = v;
        return;
    }
    const long long p = local - I.n_c;
    const int nu = (int)(p / I.N_q);
    const long long q = p - (long long)nu * I.N_q;
    reinterpret_cast<R *>(Q.popN)[I.N_off + (long long)nu * I.N_q_pad + q] = v;
    if (I.M > 0) {
        const int a = Q.compact[I.compact_base + p];
        if (a >= 0) reinterpret_cast<R *>(Q.popP)[I.P_off + a] = v;
    }
}

}  // namespace rtbte
