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
    const int *eoff, *poff, *ppoff;  // item offsets per row (absolute item ids)
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

template <class R>
__device__ __forceinline__ double item_sum(const RowParams &Q, int i0, int i1) {
    const R *P = reinterpret_cast<const R *>(Q.partials);
    double acc = 0.0;
    for (int it = i0; it < i1; ++it) acc += (double)P[2 * it] + (double)P[2 * it + 1];
    return acc;
}

// RHS value of row `local` of instance I for the selected parts.
template <class R>
__device__ __forceinline__ double row_value(const RowParams &Q, const InstDev &I, long long local, unsigned parts) {
    if (local < I.n_c) {
        if (!(parts & RTBTE_EPH)) return 0.0;
        const int d = (int)local;
        double acc = 0.0;
        for (int nu = 0; nu < I.nmodes; ++nu) {
            const int *o = Q.eoff + I.eoff_base + (long long)nu * (I.n_c + 1);
            acc += item_sum<R>(Q, o[d], o[d + 1]);
        }
        return -acc;
    }
    const long long p = local - I.n_c;
    double acc = 0.0;
    if (parts & RTBTE_PHE) {
        const int *o = Q.poff + I.poff_base;
        acc += item_sum<R>(Q, o[p], o[p + 1]);
    }
    if ((parts & RTBTE_PHPH) && I.M > 0) {
        const int a = Q.compact[I.compact_base + p];
        if (a >= 0) {
            const int *o = Q.ppoff + I.ppoff_base;
            acc += item_sum<R>(Q, o[a], o[a + 1]);
        }
    }
    return -acc;
}

// Store component value v of row `local` into the population copies read by the RHS.
template <class R>
__device__ __forceinline__ void write_pops(const RowParams &Q, const InstDev &I, long long local, double v) {
    if (local < I.n_c) {
        reinterpret_cast<R *>(Q.popf)[I.f_off + local] = (R)v;
        return;
    }
    const long long p = local - I.n_c;
    const int nu = (int)(p / I.N_q);
    const long long q = p - (long long)nu * I.N_q;
    reinterpret_cast<R *>(Q.popN)[I.N_off + (long long)nu * I.N_q_pad + q] = (R)v;
    if (I.M > 0) {
        const int a = Q.compact[I.compact_base + p];
        if (a >= 0) reinterpret_cast<R *>(Q.popP)[I.P_off + a] = (R)v;
    }
}

}  // namespace rtbte
