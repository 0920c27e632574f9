// surrogate.cu -- neural-operator stand-in for the ph-ph collision integral.
//
// The paper has no learned component; this file is the learned part of this library: a
// small periodic-convolution network maps the phonon populations of the ph-ph sub-lattice
// (one channel per branch) to I^{ph-ph} (Eq. ph-ph) on that sub-lattice.  It is trained on
// (population, exact integral) pairs collected from the library's own exact evaluations,
// and the MRI integrator uses it in the slow stage in control-variate form with the exact
// kernel as periodic judge and fallback (integrate.cu).
//
// Network (per sample, points p on the nq_s x nq_s sub-lattice, periodic):
//   x = (N - mu)/sd;  h_l = tanh(conv3x3(h_{l-1}) + b_l), l = 1..4 (C -> W -> W -> W -> W);
//   h5 = tanh(h4 M1 + c1);  out = h5 M2 + c2;  I = out * so.
// Every product is a GEMM on BF16 operands with FP32 accumulation on the tensor cores
// (mma.sync m16n8k16); convolutions are GEMMs over im2col columns (k = tap*C_in + c_in,
// tap = (dy+1)*3 + (dx+1)), their input gradients are gathers of the column gradients
// (col2im), weight gradients use split-K with a fixed-order reduction.  FP32 master
// weights, Adam, FP32 activations for the tanh derivatives.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "internal.cuh"
#include "umma.cuh"

using namespace rtbte;

namespace {

typedef __nv_bfloat16 bf16;
constexpr int kBM = 64, kBN = 64, kBK = 32, kGemmThreads = 128;
constexpr int kLayers = 4;

// C[M x N] (+)= op(A)[M x K] * op(B)[K x N]; A(m,k) = TA ? A[k*lda+m] : A[m*lda+k],
// B(k,n) = TB ? B[n*ldb+k] : B[k*ldb+n].  Split-K: blockIdx.z takes K range z, writing to
// C + z*M*ldc.  Epilogue (split 1 only): + bias[n], tanh if act, BF16 copy if Cb.
template <bool TA, bool TB>
__global__ void __launch_bounds__(kGemmThreads) gemm_bf16(const bf16 *A, int lda, const bf16 *B, int ldb, float *C,
                                                          int ldc, int M, int N, int K, int kchunk, const float *bias,
                                                          int act, bf16 *Cb) {
    __shared__ __align__(16) bf16 As[kBM][kBK + 8];
    __shared__ __align__(16) bf16 Bt[kBN][kBK + 8];  // transposed: n-major, k contiguous
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = kb; k0 < ke; k0 += kBK) {
        for (int e = tid; e < kBM * kBK; e += kGemmThreads) {
            int m, k;
            if (TA) { k = e / kBM; m = e % kBM; } else { m = e / kBK; k = e % kBK; }
            const int gm = m0 + m, gk = k0 + k;
            As[m][k] = (gm < M && gk < ke) ? (TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk]) : zero;
        }
        for (int e = tid; e < kBN * kBK; e += kGemmThreads) {
            int n, k;
            if (TB) { n = e / kBK; k = e % kBK; } else { k = e / kBN; n = e % kBN; }
            const int gn = n0 + n, gk = k0 + k;
            Bt[n][k] = (gn < N && gk < ke) ? (TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn]) : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            unsigned a[2][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm * 32 + mi * 16 + g;
                a[mi][0] = *reinterpret_cast<const unsigned *>(&As[r][kk + 2 * t4]);
                a[mi][1] = *reinterpret_cast<const unsigned *>(&As[r + 8][kk + 2 * t4]);
                a[mi][2] = *reinterpret_cast<const unsigned *>(&As[r][kk + 2 * t4 + 8]);
                a[mi][3] = *reinterpret_cast<const unsigned *>(&As[r + 8][kk + 2 * t4 + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int c = wn * 32 + ni * 8 + g;
                b[ni][0] = *reinterpret_cast<const unsigned *>(&Bt[c][kk + 2 * t4]);
                b[ni][1] = *reinterpret_cast<const unsigned *>(&Bt[c][kk + 2 * t4 + 8]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                        "{%0,%1,%2,%3};\n"
                        : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
                        : "r"(a[mi][0]), "r"(a[mi][1]), "r"(a[mi][2]), "r"(a[mi][3]), "r"(b[ni][0]), "r"(b[ni][1]));
        }
        __syncthreads();
    }
    float *Cz = C + (long long)blockIdx.z * M * ldc;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = m0 + wm * 32 + mi * 16 + g + (r >= 2 ? 8 : 0);
                const int col = n0 + wn * 32 + ni * 8 + 2 * t4 + (r & 1);
                if (row >= M || col >= N) continue;
                float v = acc[mi][ni][r];
                if (bias) v += bias[col];
                if (act) v = tanhf(v);
                Cz[(long long)row * ldc + col] = v;
                if (Cb) Cb[(long long)row * ldc + col] = __float2bfloat16(v);
            }
}

// Fixed-order sum of split-K partials: out[i] = sum_z part[z*n + i].
__global__ void sum_splits(const float *part, int splits, long long n, float *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(long long)z * n + i];
        out[i] = s;
    }
}

// im2col with periodic padding: col[p][tap*C + c] = act[b, (y+dy)%ny, (x+dx)%nx, c], zero pad to kpad.
__global__ void im2col(const bf16 *act, int C, int ny, int nx, long long P, bf16 *col, int kpad) {
    const long long total = P * kpad;
    const long long per = (long long)ny * nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / kpad;
        const int k = (int)(i - p * kpad);
        bf16 v = __float2bfloat16(0.f);
        if (k < 9 * C) {
            const int tap = k / C, c = k - tap * C;
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            const long long b = p / per;
            const int yx = (int)(p - b * per), y = yx / nx, x = yx - y * nx;
            const int ys = (y + dy + ny) % ny, xs = (x + dx + nx) % nx;
            v = act[(b * per + (long long)ys * nx + xs) * C + c];
        }
        col[i] = v;
    }
}

// col2im (gather form): g_act[b,y,x,c] = sum_tap gcol[b, (y-dy)%ny, (x-dx)%nx][tap*C + c]
__global__ void col2im(const float *gcol, int C, int ny, int nx, long long P, int kpad, float *gact) {
    const long long total = P * C;
    const long long per = (long long)ny * nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C;
        const int c = (int)(i - p * C);
        const long long b = p / per;
        const int yx = (int)(p - b * per), y = yx / nx, x = yx - y * nx;
        float s = 0.f;
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            const int ys = (y - dy + ny) % ny, xs = (x - dx + nx) % nx;
            s += gcol[(b * per + (long long)ys * nx + xs) * kpad + tap * C + c];
        }
        gact[i] = s;
    }
}

// gz = g_act * (1 - a^2) in FP32 and BF16
__global__ void tanh_back(const float *ga, const float *a, long long n, float *gz, bf16 *gzb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = ga[i] * (1.f - a[i] * a[i]);
        gz[i] = v;
        gzb[i] = __float2bfloat16(v);
    }
}

// column sums of G [M x N] (bias gradients), one block per column, fixed order
__global__ void col_sums(const float *G, long long M, int N, float *out) {
    __shared__ float red[256];
    const int col = blockIdx.x;
    float s = 0.f;
    for (long long r = threadIdx.x; r < M; r += blockDim.x) s += G[r * N + col];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[col] = red[0];
}

// mean-square loss: g = 2 (out - t)/n, per-block partial losses
__global__ void mse(const float *out, const float *t, long long n, float *g, float *part) {
    __shared__ float red[256];
    float s = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = out[i] - t[i];
        g[i] = 2.f * d / (float)n;
        s += d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0] / (float)n;
}

__global__ void to_bf16(const float *x, long long n, bf16 *y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

// Adam on the FP32 master weights; refresh the BF16 copy.
__global__ void adam(float *w, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                     float c1, float c2, bf16 *wb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wb[i] = __float2bfloat16(wi);
    }
}

// y (state vector) -> normalised sub-lattice input x[b][p][c] (BF16) for sample b of a batch
__global__ void gather_input(const double *y, const int *pp_full, long long yoff_N, int C, long long Pq, const float *mu,
                             const float *sd, bf16 *xb, float *xf) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Pq * C; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C;
        const int c = (int)(i - p * C);
        const float v = (float)((y[yoff_N + pp_full[(long long)c * Pq + p]] - mu[c]) / sd[c]);
        if (xb) xb[i] = __float2bfloat16(v);
        if (xf) xf[i] = v;
    }
}

// one collected pair: N and I on the sub-lattice from y and the exact slow RHS
__global__ void gather_pair(const double *y, const double *ydot, const int *pp_full, long long yoff_N, int C,
                            long long Pq, float *Nout, float *Iout) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Pq * C; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C;
        const int c = (int)(i - p * C);
        const long long r = yoff_N + pp_full[(long long)c * Pq + p];
        Nout[i] = (float)y[r];
        Iout[i] = (float)ydot[r];
    }
}

// minibatch assembly from stored pairs: x = (N - mu)/sd (BF16), t = I/so
__global__ void gather_batch(const float *Ns, const float *Is, const int *idx, int B, int C, long long Pq, const float *mu,
                             const float *sd, const float *so, bf16 *xb, float *t) {
    const long long per = Pq * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)B * per;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / per);
        const long long j = i - (long long)b * per;
        const int c = (int)(j % C);
        const long long src = (long long)idx[b] * per + j;
        xb[i] = __float2bfloat16((Ns[src] - mu[c]) / sd[c]);
        t[i] = Is[src] / so[c];
    }
}

// out (normalised) -> I = out * so scattered into phonon rows of a state-size vector
__global__ void scatter_output(const float *out, const int *pp_full, long long yoff_N, int C, long long Pq,
                               const float *so, double *dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Pq * C; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C;
        const int c = (int)(i - p * C);
        dst[yoff_N + pp_full[(long long)c * Pq + p]] = (double)out[i] * so[c];
    }
}

// control-variate value on the sub-lattice rows: dst[row(p,c)] = Eref[p*C+c] + (out - out_ref) * so[c]
// (Eref, out, out_ref in the network's [point][channel] layout)
__global__ void cv_write(const float *out, const float *out_ref, const double *Eref, const int *pp_full,
                         long long yoff_N, int C, long long Pq, const float *so, double *dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Pq * C; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C;
        const int c = (int)(i - p * C);
        dst[yoff_N + pp_full[(long long)c * Pq + p]] = Eref[i] + ((double)out[i] - (double)out_ref[i]) * so[c];
    }
}

// Judge: per-block partial sums of |cv - exact|^2 and |exact|^2 over the sub-lattice rows, where
// cv = Eref + (out - out_ref) * so; then (exact, out) become the new reference, in place.
__global__ void judge_cv(const float *out, float *out_ref, double *Eref, const double *exact, const int *pp_full,
                         long long yoff_N, int C, long long Pq, const float *so, double *part) {
    __shared__ double r0[256], r1[256];
    double s0 = 0, s1 = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Pq * C; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C;
        const int c = (int)(i - p * C);
        const double ex = exact[yoff_N + pp_full[(long long)c * Pq + p]];
        const double cv = Eref[i] + ((double)out[i] - (double)out_ref[i]) * so[c];
        s0 += (cv - ex) * (cv - ex);
        s1 += ex * ex;
        Eref[i] = ex;
        out_ref[i] = out[i];
    }
    r0[threadIdx.x] = s0;
    r1[threadIdx.x] = s1;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            r0[threadIdx.x] += r0[threadIdx.x + o];
            r1[threadIdx.x] += r1[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = r0[0];
        part[2 * blockIdx.x + 1] = r1[0];
    }
}

// difference loss for pairs (sample b, sample b + B): d = (out_b - out_{b+B}) - (t_b - t_{b+B});
// loss = mean(d^2) over the first half; g_b = 2d/n, g_{b+B} = -2d/n
__global__ void mse_diff(const float *out, const float *t, long long n, float *g, float *part) {
    __shared__ float red[256];
    float s = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = (out[i] - out[i + n]) - (t[i] - t[i + n]);
        g[i] = 2.f * d / (float)n;
        g[i + n] = -2.f * d / (float)n;
        s += d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0] / (float)n;
}

// BF16 transposed copy of a [K x N] FP32 master matrix: Wt[n*K + k] = W[k*N + n]
__global__ void transpose_bf16(const float *W, int K, int N, bf16 *Wt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)K * N;
         i += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(i / K), k = (int)(i - (long long)n * K);
        Wt[i] = __float2bfloat16(W[(long long)k * N + n]);
    }
}

// ---- fused single-sample inference (width 64) -------------------------------------------
// One CTA computes kIM points x 64 channels of a conv layer as one GEMM over K = 9*C_in
// (zero-padded to KP): the whole A block (the 3x3 periodic neighbourhoods, gathered from the
// previous activation, or from the state vector y for the first layer) and the whole
// transposed weight block are staged in shared memory by one burst of 16-byte cp.async
// copies, so the K loop runs from shared memory with a single wait.  The last layer also
// applies the pointwise MLP and writes the control-variate value.
constexpr int kIM = 32, kIW = 64, kIThreads = 128;

struct InferArgs {
    const bf16 *act_in;  // [Pq][64] previous activation (middle and last layers)
    const double *y;     // state vector (first layer)
    const int *pp_full;  // [C][Pq] state row (minus yN) of sub-lattice point p, branch c
    long long yN, Pq;
    const float *mu, *sd, *so;
    int C, KP, ny, nx;
    const bf16 *Wt;      // [64][KP] transposed BF16 conv weights
    const float *bias;   // [64]
    bf16 *act_out;       // [Pq][64] (first and middle layers)
    const bf16 *M1t;     // [64][64] transposed BF16 M1
    const float *c1;     // [64]
    const bf16 *M2;      // [64][C] BF16
    const float *c2;     // [C]
    float *out;          // [Pq][C] network output (normalised)
    const float *out_ref;
    const double *Eref;  // [Pq][C]
    double *dst;         // state-size vector receiving the control-variate value (may be null)
};

__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}

__device__ __forceinline__ long long neighbour(long long p, int tap, int ny, int nx) {
    const int y = (int)(p / nx), x = (int)(p - (long long)y * nx);
    const int ys = (y + tap / 3 - 1 + ny) % ny, xs = (x + tap % 3 - 1 + nx) % nx;
    return (long long)ys * nx + xs;
}

// 4 warps: warp w covers rows (w>>1)*16..+16 and columns (w&1)*32..+32 of a kIM x 64 tile;
// A [kIM][lda], Bt [64][lda] (k contiguous), K a multiple of 16.
__device__ __forceinline__ void tile_mma(const bf16 *A, const bf16 *Bt, int lda, int K, float acc[4][4]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t4 = lane & 3;
    const int r0 = (warp >> 1) * 16 + g, c0 = (warp & 1) * 32 + g;
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[ni][r] = 0.f;
    for (int kk = 0; kk < K; kk += 16) {
        unsigned a[4];
        a[0] = *reinterpret_cast<const unsigned *>(A + r0 * lda + kk + 2 * t4);
        a[1] = *reinterpret_cast<const unsigned *>(A + (r0 + 8) * lda + kk + 2 * t4);
        a[2] = *reinterpret_cast<const unsigned *>(A + r0 * lda + kk + 2 * t4 + 8);
        a[3] = *reinterpret_cast<const unsigned *>(A + (r0 + 8) * lda + kk + 2 * t4 + 8);
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const bf16 *b = Bt + (c0 + ni * 8) * lda + kk + 2 * t4;
            const unsigned b0 = *reinterpret_cast<const unsigned *>(b);
            const unsigned b1 = *reinterpret_cast<const unsigned *>(b + 8);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(acc[ni][0]), "+f"(acc[ni][1]), "+f"(acc[ni][2]), "+f"(acc[ni][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
        }
    }
}

// MODE 0: first layer (input from y), 1: middle layer, 2: last conv layer + MLP + outputs
template <int MODE>
__global__ void __launch_bounds__(kIThreads) infer_conv(InferArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lda = a.KP + 8;
    bf16 *As = reinterpret_cast<bf16 *>(smem);
    bf16 *Bs = As + kIM * lda;
    const int tid = threadIdx.x;
    const long long p0 = (long long)blockIdx.x * kIM;
    const int kch = a.KP / 8;  // 16-byte chunks per row
    for (int e = tid; e < kIW * kch; e += kIThreads) {
        const int n = e / kch, ch = e - n * kch;
        cp16(Bs + n * lda + ch * 8, a.Wt + (long long)n * a.KP + ch * 8);
    }
    if (MODE == 0) {
        // gathers from y through pp_full: issue a batch of independent index loads, then the
        // value loads, so each thread waits for two memory round trips per batch, not per element
        constexpr int kB = 8;
        const int K9 = 9 * a.C, total = kIM * a.KP;
        for (int e0 = tid; e0 < total; e0 += kB * kIThreads) {
            int row[kB];
            int ci_[kB];
#pragma unroll
            for (int j = 0; j < kB; ++j) {
                const int e = e0 + j * kIThreads;
                row[j] = -1;
                ci_[j] = 0;
                if (e < total) {
                    const int m = e / a.KP, k = e - m * a.KP;
                    const long long p = p0 + m;
                    if (p < a.Pq && k < K9) {
                        const int tap = k / a.C, ci = k - tap * a.C;
                        ci_[j] = ci;
                        row[j] = a.pp_full[(long long)ci * a.Pq + neighbour(p, tap, a.ny, a.nx)];
                    }
                }
            }
            double yv[kB];
#pragma unroll
            for (int j = 0; j < kB; ++j) yv[j] = row[j] >= 0 ? a.y[a.yN + row[j]] : 0.0;
#pragma unroll
            for (int j = 0; j < kB; ++j) {
                const int e = e0 + j * kIThreads;
                if (e >= total) continue;
                const float v = row[j] >= 0 ? (float)((yv[j] - a.mu[ci_[j]]) / a.sd[ci_[j]]) : 0.f;
                As[(e / a.KP) * lda + (e % a.KP)] = __float2bfloat16(v);
            }
        }
    } else {
        for (int e = tid; e < kIM * 9 * (kIW / 8); e += kIThreads) {
            const int m = e / (9 * (kIW / 8)), r = e - m * 9 * (kIW / 8);
            const int tap = r / (kIW / 8), ch = r - tap * (kIW / 8);
            const long long p = p0 + m;
            bf16 *d = As + m * lda + tap * kIW + ch * 8;
            if (p < a.Pq)
                cp16(d, a.act_in + neighbour(p, tap, a.ny, a.nx) * kIW + ch * 8);
            else
                *reinterpret_cast<uint4 *>(d) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    bf16 *M1s = Bs + kIW * lda, *H4 = M1s + kIW * 72;
    float *H5 = reinterpret_cast<float *>(H4 + kIM * 72), *M2s = H5 + kIM * 65;
    if (MODE == 2) {
        for (int e = tid; e < kIW * 8; e += kIThreads) cp16(M1s + (e >> 3) * 72 + (e & 7) * 8, a.M1t + e * 8);
        for (int e = tid; e < kIW * a.C; e += kIThreads) M2s[e] = __bfloat162float(a.M2[e]);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    float acc[4][4];
    tile_mma(As, Bs, lda, a.KP, acc);
    const int lane = tid & 31, warp = tid >> 5, g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = (warp >> 1) * 16 + g + h * 8, col = (warp & 1) * 32 + ni * 8 + 2 * t4;
            __nv_bfloat162 v;
            v.x = __float2bfloat16(tanhf(acc[ni][2 * h] + a.bias[col]));
            v.y = __float2bfloat16(tanhf(acc[ni][2 * h + 1] + a.bias[col + 1]));
            if (MODE == 2) {
                *reinterpret_cast<__nv_bfloat162 *>(H4 + row * 72 + col) = v;
            } else if (p0 + row < a.Pq) {
                *reinterpret_cast<__nv_bfloat162 *>(a.act_out + (p0 + row) * kIW + col) = v;
            }
        }
    if (MODE != 2) return;
    __syncthreads();
    tile_mma(H4, M1s, 72, kIW, acc);
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int row = (warp >> 1) * 16 + g + (r >> 1) * 8, col = (warp & 1) * 32 + ni * 8 + 2 * t4 + (r & 1);
            H5[row * 65 + col] = __bfloat162float(__float2bfloat16(tanhf(acc[ni][r] + a.c1[col])));
        }
    __syncthreads();
    for (int e = tid; e < kIM * a.C; e += kIThreads) {
        const int r = e / a.C, c = e - r * a.C;
        const long long p = p0 + r;
        if (p >= a.Pq) continue;
        float sacc = 0.f;
        for (int j = 0; j < kIW; ++j) sacc = fmaf(H5[r * 65 + j], M2s[j * a.C + c], sacc);
        const float o = sacc + a.c2[c];
        const long long i = p * a.C + c;
        a.out[i] = o;
        if (a.dst)
            a.dst[a.yN + a.pp_full[(long long)c * a.Pq + p]] = a.Eref[i] + ((double)o - (double)a.out_ref[i]) * a.so[c];
    }
}

size_t infer_smem(int KP, int mode) {
    size_t b = sizeof(bf16) * (size_t)(kIM + kIW) * (KP + 8);
    if (mode == 2) b += sizeof(bf16) * (kIW + kIM) * 72 + sizeof(float) * (kIM * 65 + kIW * 16);
    return b;
}

int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

}  // namespace

// ---------------------------------------------------------------------------------------
struct rtbte_surrogate {
    rtbte_ctx *ctx = nullptr;
    int inst = 0, C = 0, width = 0, ny = 0, nx = 0;
    long long Pq = 0;  // points per sample
    int capacity = 0, count = 0, max_batch = 0;
    int cin[kLayers], kpad[kLayers];
    long long off_W[kLayers], off_b[kLayers], off_M1 = 0, off_c1 = 0, off_M2 = 0, off_c2 = 0, nparam = 0;
    DevBuf w, wb, g, m, v, stats, ppfull;  // params FP32/BF16, grads, Adam moments, mu|sd|so
    DevBuf Ns, Is, idx;                    // collected pairs, minibatch indices
    DevBuf xb, t, cols[kLayers], acts[kLayers + 1], actb[kLayers + 1], out, gout, goutb, ga, gz, gzb, gcol, split,
        lossp, ydot;
    DevBuf Eref, out_ref, normp;  // control-variate reference [Pq][C]: exact value, network output
    DevBuf wbt, a0, a1;           // transposed BF16 weights and activations of the fused inference path
    DevBuf wtt, tcerr;            // K-major BF16 weights of the tensor-core GEMMs (W_l^T, M1^T, M2^T); error word
    long long off_tt[kLayers + 2] = {0, 0, 0, 0, 0, 0};
    int engine = 0;               // 0: tcgen05 GEMMs where both operands are K-major; 1: mma.sync everywhere
    long long off_t[kLayers + 1] = {0, 0, 0, 0, 0};
    bool has_ref = false, fused = false, smem_set = false;
    std::vector<int> traj;        // trajectory id of each collected pair
    long long adam_t = 0;
    bool stats_set = false;
    float mu[16], sd[16], so[16];
    std::mt19937_64 rng;
    std::string err;
};

namespace {

int sfail(rtbte_surrogate *s, int code, const char *msg) {
    if (s) s->err = msg;
    return code;
}

#define S_CUDA(s, call)                                            \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) {                                   \
            cudaGetLastError();                                    \
            if (s) s->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
            return RTBTE_E_CUDA;                                   \
        }                                                          \
    } while (0)

int salloc(rtbte_surrogate *s, DevBuf &b, size_t bytes) {
    b.release();
    S_CUDA(s, cudaMalloc(&b.p, std::max<size_t>(bytes, 16)));
    b.bytes = bytes;
    return RTBTE_OK;
}

template <bool TA, bool TB>
int gemm(rtbte_surrogate *s, const bf16 *A, int lda, const bf16 *B, int ldb, float *C, int ldc, int M, int N, int K,
         const float *bias, int act, bf16 *Cb, int splits = 1) {
    cudaStream_t st = s->ctx->stream;
    if (splits <= 1) {
        dim3 grid((M + kBM - 1) / kBM, (N + kBN - 1) / kBN, 1);
        gemm_bf16<TA, TB><<<grid, kGemmThreads, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K, K, bias, act, Cb);
    } else {
        int kchunk = (K + splits - 1) / splits;
        kchunk = (kchunk + kBK - 1) / kBK * kBK;
        splits = (K + kchunk - 1) / kchunk;
        dim3 grid((M + kBM - 1) / kBM, (N + kBN - 1) / kBN, splits);
        float *part = s->split.as<float>();
        gemm_bf16<TA, TB><<<grid, kGemmThreads, 0, st>>>(A, lda, B, ldb, part, ldc, M, N, K, kchunk, nullptr, 0, nullptr);
        sum_splits<<<blocks_for((long long)M * ldc), 256, 0, st>>>(part, splits, (long long)M * ldc, C);
    }
    S_CUDA(s, cudaGetLastError());
    s->ctx->launches += splits <= 1 ? 1 : 2;
    return RTBTE_OK;
}

// ---- tcgen05 GEMMs ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// TMA map of a K-major BF16 matrix [rows x cols] (row stride ld elements), boxes of 64 columns x
// box_rows rows, 128-byte swizzle, zero fill outside
bool kmajor_map(CUtensorMap *m, const bf16 *ptr, long long rows, long long cols, long long ld, int box_rows) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(bf16)};
    const cuuint32_t box[2] = {(cuuint32_t)umma::kTK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C[M x N] = A[M x K] B[N x K]^T (+ bias, tanh, BF16 copy) on the tensor cores, A and B K-major
int gemm_tc(rtbte_surrogate *s, const bf16 *A, int lda, const bf16 *B, int ldb, float *C, int ldc, int M, int N, int K,
            const float *bias, int act, bf16 *Cb) {
    const int bn_full = (N + 15) / 16 * 16;
    const int bn = std::min(bn_full, 256);
    CUtensorMap ta, tb;
    if ((lda * (int)sizeof(bf16)) % 16 || (ldb * (int)sizeof(bf16)) % 16 || !kmajor_map(&ta, A, M, K, lda, umma::kTM) ||
        !kmajor_map(&tb, B, N, K, ldb, bn))
        return sfail(s, RTBTE_E_UNSUPPORTED, "tensor-core GEMM: operand layout not expressible as a TMA map");
    umma::Args a;
    a.M = M;
    a.N = N;
    a.K = K;
    a.bn = bn;
    a.ldc = ldc;
    a.act = act;
    a.bias = bias;
    a.C = C;
    a.Cb = Cb;
    a.err = s->tcerr.as<int>();
    a.a_mn = a.b_mn = 0;
    a.k_base = 0;
    a.c_split = 0;
    const dim3 grid((M + umma::kTM - 1) / umma::kTM, (N + bn - 1) / bn);
    const size_t sm = umma::smem_bytes(bn);
    cudaStream_t st = s->ctx->stream;
    static bool attr_set = false;  // the shared-memory limit is a per-function attribute: set once
    if (!attr_set) {
        const void *fns[4] = {(const void *)umma::gemm_tc<32, 4>, (const void *)umma::gemm_tc<64, 4>,
                              (const void *)umma::gemm_tc<128, 4>, (const void *)umma::gemm_tc<256, 2>};
        for (const void *f : fns) S_CUDA(s, allow_max_dynamic_smem(f));
        attr_set = true;
    }
    static_assert(umma::kTM * umma::kTK * 2 + 128 * umma::kTK * 2 <= 32768, "four stages for bn <= 128");
    if (bn <= 32) umma::gemm_tc<32, 4><<<grid, umma::kThreads, sm, st>>>(ta, tb, a);
    else if (bn <= 64) umma::gemm_tc<64, 4><<<grid, umma::kThreads, sm, st>>>(ta, tb, a);
    else if (bn <= 128) umma::gemm_tc<128, 4><<<grid, umma::kThreads, sm, st>>>(ta, tb, a);
    else umma::gemm_tc<256, 2><<<grid, umma::kThreads, sm, st>>>(ta, tb, a);
    S_CUDA(s, cudaGetLastError());
    s->ctx->launches++;
    return RTBTE_OK;
}

// C[M x N] = A^T B on the tensor cores for A stored [K][M] (row stride lda) and B stored [K][N]
// (row stride ldb), both MN-major, N a multiple of 64: K split over CTAs in multiples of 64, the
// partial products summed in a fixed order (the weight gradients, a contraction over points)
int gemm_tc_mn(rtbte_surrogate *s, const bf16 *A, int lda, const bf16 *B, int ldb, float *C, int ldc, int M, int N,
               int K) {
    if (N % 64 || N > 256) return sfail(s, RTBTE_E_UNSUPPORTED, "tensor-core GEMM: MN-major N must be 64..256 by 64");
    CUtensorMap ta, tb;
    if ((lda * (int)sizeof(bf16)) % 16 || (ldb * (int)sizeof(bf16)) % 16 || !kmajor_map(&ta, A, K, M, lda, 64) ||
        !kmajor_map(&tb, B, K, N, ldb, 64))
        return sfail(s, RTBTE_E_UNSUPPORTED, "tensor-core GEMM: operand layout not expressible as a TMA map");
    const int mt = (M + umma::kTM - 1) / umma::kTM;
    // about two CTAs per SM, at most 64 slices, each a whole number of 64-wide K slices
    const int want = std::max(1, std::min(64, (2 * s->ctx->num_sms + mt - 1) / mt));
    long long kc = ((long long)K + want - 1) / want;
    kc = (kc + umma::kTK - 1) / umma::kTK * umma::kTK;
    const int splits = (int)((K + kc - 1) / kc);
    umma::Args a{};
    a.M = M;
    a.N = N;
    a.K = (int)kc;
    a.bn = N;
    a.ldc = ldc;
    a.act = 0;
    a.C = splits > 1 ? s->split.as<float>() : C;
    a.err = s->tcerr.as<int>();
    a.a_mn = a.b_mn = 1;
    a.k_base = 0;
    a.c_split = (long long)M * ldc;
    const dim3 grid(mt, 1, splits);
    cudaStream_t st = s->ctx->stream;
    if (N <= 64) umma::gemm_tc<64, 4><<<grid, umma::kThreads, umma::smem_bytes(64), st>>>(ta, tb, a);
    else if (N <= 128) umma::gemm_tc<128, 4><<<grid, umma::kThreads, umma::smem_bytes(128), st>>>(ta, tb, a);
    else umma::gemm_tc<256, 2><<<grid, umma::kThreads, umma::smem_bytes(N), st>>>(ta, tb, a);
    S_CUDA(s, cudaGetLastError());
    s->ctx->launches++;
    if (splits > 1) {
        sum_splits<<<blocks_for((long long)M * ldc), 256, 0, st>>>(s->split.as<float>(), splits, (long long)M * ldc, C);
        S_CUDA(s, cudaGetLastError());
        s->ctx->launches++;
    }
    return RTBTE_OK;
}

// K-major BF16 copies of the weights for the tensor-core forward GEMMs, refreshed after every
// change of the master weights: W_l^T [w x kpad_l], M1^T [w x w], M2^T [C x w]
int refresh_training_layout(rtbte_surrogate *s) {
    if (s->engine != 0) return RTBTE_OK;
    cudaStream_t st = s->ctx->stream;
    bf16 *wt = s->wtt.as<bf16>();
    const float *w = s->w.as<float>();
    for (int l = 0; l < kLayers; ++l)
        transpose_bf16<<<blocks_for((long long)s->kpad[l] * s->width), 256, 0, st>>>(w + s->off_W[l], s->kpad[l],
                                                                                   s->width, wt + s->off_tt[l]);
    transpose_bf16<<<blocks_for((long long)s->width * s->width), 256, 0, st>>>(w + s->off_M1, s->width, s->width,
                                                                             wt + s->off_tt[kLayers]);
    transpose_bf16<<<blocks_for((long long)s->width * s->C), 256, 0, st>>>(w + s->off_M2, s->width, s->C,
                                                                         wt + s->off_tt[kLayers + 1]);
    S_CUDA(s, cudaGetLastError());
    s->ctx->launches += kLayers + 2;
    return RTBTE_OK;
}

// the error word of the tensor-core GEMMs (a bounded wait that gave up); synchronises
int check_tc(rtbte_surrogate *s) {
    if (s->engine != 0) return RTBTE_OK;
    int e = 0;
    S_CUDA(s, cudaMemcpyAsync(&e, s->tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, s->ctx->stream));
    S_CUDA(s, cudaStreamSynchronize(s->ctx->stream));
    if (e) return sfail(s, RTBTE_E_TIMEOUT, "tensor-core GEMM: a bounded mbarrier wait gave up");
    return RTBTE_OK;
}

// forward of B samples whose normalised input is in s->xb ([B*Pq][C] BF16); output FP32 in s->out
int forward(rtbte_surrogate *s, int B) {
    cudaStream_t st = s->ctx->stream;
    const long long P = (long long)B * s->Pq;
    const bf16 *in = s->xb.as<bf16>();
    int C = s->C, rc;
    for (int l = 0; l < kLayers; ++l) {
        im2col<<<blocks_for(P * s->kpad[l]), 256, 0, st>>>(in, C, s->ny, s->nx, P, s->cols[l].as<bf16>(), s->kpad[l]);
        S_CUDA(s, cudaGetLastError());
        s->ctx->launches++;
        if (s->engine == 0)
            rc = gemm_tc(s, s->cols[l].as<bf16>(), s->kpad[l], s->wtt.as<bf16>() + s->off_tt[l], s->kpad[l],
                         s->acts[l + 1].as<float>(), s->width, (int)P, s->width, s->kpad[l],
                         s->w.as<float>() + s->off_b[l], 1, s->actb[l + 1].as<bf16>());
        else
            rc = gemm<false, false>(s, s->cols[l].as<bf16>(), s->kpad[l], s->wb.as<bf16>() + s->off_W[l], s->width,
                                    s->acts[l + 1].as<float>(), s->width, (int)P, s->width, s->kpad[l],
                                    s->w.as<float>() + s->off_b[l], 1, s->actb[l + 1].as<bf16>());
        if (rc) return rc;
        in = s->actb[l + 1].as<bf16>();
        C = s->width;
    }
    // pointwise MLP: h5 = tanh(h4 M1 + c1) (reuses acts[0]), out = h5 M2 + c2
    if (s->engine == 0) {
        if ((rc = gemm_tc(s, s->actb[kLayers].as<bf16>(), s->width, s->wtt.as<bf16>() + s->off_tt[kLayers], s->width,
                          s->acts[0].as<float>(), s->width, (int)P, s->width, s->width, s->w.as<float>() + s->off_c1, 1,
                          s->actb[0].as<bf16>())))
            return rc;
        return gemm_tc(s, s->actb[0].as<bf16>(), s->width, s->wtt.as<bf16>() + s->off_tt[kLayers + 1], s->width,
                       s->out.as<float>(), s->C, (int)P, s->C, s->width, s->w.as<float>() + s->off_c2, 0, nullptr);
    }
    if ((rc = gemm<false, false>(s, s->actb[kLayers].as<bf16>(), s->width, s->wb.as<bf16>() + s->off_M1, s->width,
                                 s->acts[0].as<float>(), s->width, (int)P, s->width, s->width,
                                 s->w.as<float>() + s->off_c1, 1, s->actb[0].as<bf16>())))
        return rc;
    return gemm<false, false>(s, s->actb[0].as<bf16>(), s->width, s->wb.as<bf16>() + s->off_M2, s->C,
                              s->out.as<float>(), s->C, (int)P, s->C, s->width, s->w.as<float>() + s->off_c2, 0,
                              nullptr);
}

// loss and gradients (FP32, s->g) for targets s->t of the B samples in s->xb
int loss_grad(rtbte_surrogate *s, int B, float *loss, bool diff = false) {
    cudaStream_t st = s->ctx->stream;
    int rc;
    if ((rc = forward(s, B))) return rc;
    const long long P = (long long)B * s->Pq, nout = P * s->C;
    const int nb = blocks_for(diff ? nout / 2 : nout);
    if (diff)  // samples b and b + B/2 form a pair
        mse_diff<<<nb, 256, 0, st>>>(s->out.as<float>(), s->t.as<float>(), nout / 2, s->gout.as<float>(),
                                     s->lossp.as<float>());
    else
        mse<<<nb, 256, 0, st>>>(s->out.as<float>(), s->t.as<float>(), nout, s->gout.as<float>(), s->lossp.as<float>());
    to_bf16<<<nb, 256, 0, st>>>(s->gout.as<float>(), nout, s->goutb.as<bf16>());
    S_CUDA(s, cudaGetLastError());
    s->ctx->launches += 2;
    float *g = s->g.as<float>();
    const int Wd = s->width;
    const int splitsP = (int)std::min<long long>(64, std::max<long long>(1, P / 1024));
    // out = h5 M2 + c2
    if ((rc = gemm<true, false>(s, s->actb[0].as<bf16>(), Wd, s->goutb.as<bf16>(), s->C, g + s->off_M2, s->C, Wd,
                                s->C, (int)P, nullptr, 0, nullptr, splitsP)))
        return rc;
    col_sums<<<s->C, 256, 0, st>>>(s->gout.as<float>(), P, s->C, g + s->off_c2);
    // g_h5 = g_out M2^T; gz5 = g_h5 (1 - h5^2)
    if ((rc = gemm<false, true>(s, s->goutb.as<bf16>(), s->C, s->wb.as<bf16>() + s->off_M2, s->C, s->ga.as<float>(),
                                Wd, (int)P, Wd, s->C, nullptr, 0, nullptr)))
        return rc;
    tanh_back<<<blocks_for(P * Wd), 256, 0, st>>>(s->ga.as<float>(), s->acts[0].as<float>(), P * Wd, s->gz.as<float>(),
                                                   s->gzb.as<bf16>());
    const bool tc_mn = s->engine == 0 && Wd % 64 == 0;  // weight gradients on the tensor cores (MN-major operands)
    if (tc_mn)
        rc = gemm_tc_mn(s, s->actb[kLayers].as<bf16>(), Wd, s->gzb.as<bf16>(), Wd, g + s->off_M1, Wd, Wd, Wd, (int)P);
    else
        rc = gemm<true, false>(s, s->actb[kLayers].as<bf16>(), Wd, s->gzb.as<bf16>(), Wd, g + s->off_M1, Wd, Wd, Wd,
                               (int)P, nullptr, 0, nullptr, splitsP);
    if (rc) return rc;
    col_sums<<<Wd, 256, 0, st>>>(s->gz.as<float>(), P, Wd, g + s->off_c1);
    // g_h4 = gz5 M1^T (M1 itself is the K-major [n][k] operand)
    if (s->engine == 0)
        rc = gemm_tc(s, s->gzb.as<bf16>(), Wd, s->wb.as<bf16>() + s->off_M1, Wd, s->ga.as<float>(), Wd, (int)P, Wd, Wd,
                     nullptr, 0, nullptr);
    else
        rc = gemm<false, true>(s, s->gzb.as<bf16>(), Wd, s->wb.as<bf16>() + s->off_M1, Wd, s->ga.as<float>(), Wd,
                               (int)P, Wd, Wd, nullptr, 0, nullptr);
    if (rc) return rc;
    for (int l = kLayers - 1; l >= 0; --l) {
        tanh_back<<<blocks_for(P * Wd), 256, 0, st>>>(s->ga.as<float>(), s->acts[l + 1].as<float>(), P * Wd,
                                                       s->gz.as<float>(), s->gzb.as<bf16>());
        // dW_l = cols_l^T gz  ([kpad x Wd]); the rows beyond 9*C_in stay zero
        if (tc_mn)
            rc = gemm_tc_mn(s, s->cols[l].as<bf16>(), s->kpad[l], s->gzb.as<bf16>(), Wd, g + s->off_W[l], Wd,
                            s->kpad[l], Wd, (int)P);
        else
            rc = gemm<true, false>(s, s->cols[l].as<bf16>(), s->kpad[l], s->gzb.as<bf16>(), Wd, g + s->off_W[l], Wd,
                                   s->kpad[l], Wd, (int)P, nullptr, 0, nullptr, splitsP);
        if (rc) return rc;
        col_sums<<<Wd, 256, 0, st>>>(s->gz.as<float>(), P, Wd, g + s->off_b[l]);
        if (l == 0) break;
        // gcol = gz W_l^T  ([P x kpad]), then col2im into the previous activation's gradient
        if (s->engine == 0)
            rc = gemm_tc(s, s->gzb.as<bf16>(), Wd, s->wb.as<bf16>() + s->off_W[l], Wd, s->gcol.as<float>(), s->kpad[l],
                         (int)P, s->kpad[l], Wd, nullptr, 0, nullptr);
        else
            rc = gemm<false, true>(s, s->gzb.as<bf16>(), Wd, s->wb.as<bf16>() + s->off_W[l], Wd, s->gcol.as<float>(),
                                   s->kpad[l], (int)P, s->kpad[l], Wd, nullptr, 0, nullptr);
        if (rc) return rc;
        col2im<<<blocks_for(P * s->cin[l]), 256, 0, st>>>(s->gcol.as<float>(), s->cin[l], s->ny, s->nx, P, s->kpad[l],
                                                          s->ga.as<float>());
    }
    S_CUDA(s, cudaGetLastError());
    s->ctx->launches += 4 + 3 * kLayers;
    if (loss) {
        std::vector<float> lp(nb);
        S_CUDA(s, cudaMemcpyAsync(lp.data(), s->lossp.p, sizeof(float) * nb, cudaMemcpyDeviceToHost, st));
        S_CUDA(s, cudaStreamSynchronize(st));
        double acc = 0;
        for (float x : lp) acc += x;
        *loss = (float)acc;
    }
    return RTBTE_OK;
}

// host <-> device parameter copies in the logical layout (W_l rows 0..9*C_in-1)
int params_io(rtbte_surrogate *s, float *host, bool to_device) {
    std::vector<float> w(s->nparam);
    if (!to_device) S_CUDA(s, cudaMemcpy(w.data(), s->w.p, sizeof(float) * s->nparam, cudaMemcpyDeviceToHost));
    long long h = 0;
    auto blk = [&](long long off, long long rows_logical, long long rows_pad, long long cols) {
        for (long long r = 0; r < rows_pad; ++r)
            for (long long c = 0; c < cols; ++c) {
                if (to_device) w[off + r * cols + c] = r < rows_logical ? host[h + r * cols + c] : 0.f;
                else if (r < rows_logical) host[h + r * cols + c] = w[off + r * cols + c];
            }
        h += rows_logical * cols;
    };
    for (int l = 0; l < kLayers; ++l) {
        blk(s->off_W[l], 9LL * s->cin[l], s->kpad[l], s->width);
        blk(s->off_b[l], 1, 1, s->width);
    }
    blk(s->off_M1, s->width, s->width, s->width);
    blk(s->off_c1, 1, 1, s->width);
    blk(s->off_M2, s->width, s->width, s->C);
    blk(s->off_c2, 1, 1, s->C);
    if (to_device) {
        S_CUDA(s, cudaMemcpy(s->w.p, w.data(), sizeof(float) * s->nparam, cudaMemcpyHostToDevice));
        to_bf16<<<blocks_for(s->nparam), 256, 0, s->ctx->stream>>>(s->w.as<float>(), s->nparam, s->wb.as<bf16>());
        S_CUDA(s, cudaGetLastError());
        S_CUDA(s, cudaStreamSynchronize(s->ctx->stream));
    }
    return RTBTE_OK;
}

// largest weight-gradient matrix (the split-K partial buffer holds 64 of them)
long long split_elems(const rtbte_surrogate *s) {
    long long e = (long long)s->width * std::max(s->width, s->C);
    for (int l = 0; l < kLayers; ++l) e = std::max(e, (long long)s->kpad[l] * s->width);
    return e;
}

int ensure_batch(rtbte_surrogate *s, int B) {
    if (B <= s->max_batch) return RTBTE_OK;
    const long long P = (long long)B * s->Pq;
    const int Wd = s->width;
    int rc;
    if ((rc = salloc(s, s->xb, sizeof(bf16) * P * s->C)) || (rc = salloc(s, s->t, sizeof(float) * P * s->C)) ||
        (rc = salloc(s, s->out, sizeof(float) * P * s->C)) || (rc = salloc(s, s->gout, sizeof(float) * P * s->C)) ||
        (rc = salloc(s, s->goutb, sizeof(bf16) * P * s->C)) || (rc = salloc(s, s->ga, sizeof(float) * P * Wd)) ||
        (rc = salloc(s, s->gz, sizeof(float) * P * Wd)) || (rc = salloc(s, s->gzb, sizeof(bf16) * P * Wd)) ||
        (rc = salloc(s, s->gcol, sizeof(float) * P * s->kpad[1])) ||
        (rc = salloc(s, s->split, sizeof(float) * 64LL * split_elems(s))) ||
        (rc = salloc(s, s->lossp, sizeof(float) * 4096)) || (rc = salloc(s, s->idx, sizeof(int) * B)))
        return rc;
    for (int l = 0; l < kLayers; ++l)
        if ((rc = salloc(s, s->cols[l], sizeof(bf16) * P * s->kpad[l]))) return rc;
    for (int l = 0; l <= kLayers; ++l)
        if ((rc = salloc(s, s->acts[l], sizeof(float) * P * Wd)) || (rc = salloc(s, s->actb[l], sizeof(bf16) * P * Wd)))
            return rc;
    s->max_batch = B;
    return RTBTE_OK;
}

int upload_stats(rtbte_surrogate *s) {
    float h[48];
    for (int c = 0; c < s->C; ++c) {
        h[c] = s->mu[c];
        h[16 + c] = s->sd[c];
        h[32 + c] = s->so[c];
    }
    S_CUDA(s, cudaMemcpy(s->stats.p, h, sizeof(h), cudaMemcpyHostToDevice));
    return RTBTE_OK;
}

// BF16 transposed weights for the fused inference path (width 64), refreshed after every
// change of the master weights
int refresh_inference(rtbte_surrogate *s) {
    if (!s->fused) return RTBTE_OK;
    cudaStream_t st = s->ctx->stream;
    bf16 *wt = s->wbt.as<bf16>();
    for (int l = 0; l < kLayers; ++l)
        transpose_bf16<<<blocks_for((long long)s->kpad[l] * kIW), 256, 0, st>>>(s->w.as<float>() + s->off_W[l],
                                                                               s->kpad[l], kIW, wt + s->off_t[l]);
    transpose_bf16<<<blocks_for(kIW * kIW), 256, 0, st>>>(s->w.as<float>() + s->off_M1, kIW, kIW, wt + s->off_t[kLayers]);
    S_CUDA(s, cudaGetLastError());
    s->ctx->launches += kLayers + 1;
    return RTBTE_OK;
}

// network output for the device state y into s->out (one sample); with dst, also the
// control-variate value on the sub-lattice rows of dst
int infer(rtbte_surrogate *s, const double *y, double *dst) {
    rtbte_ctx *ctx = s->ctx;
    const InstHost &I = ctx->inst[s->inst];
    const long long yN = I.y_off + I.d.n_c;
    const float *mu = s->stats.as<float>(), *sd = mu + 16, *so = mu + 32;
    int rc;
    if ((rc = ensure_batch(s, 1))) return rc;
    if (!s->fused) {  // general width: the training kernels with a batch of one
        gather_input<<<blocks_for(s->Pq * s->C), 256, 0, ctx->stream>>>(y, s->ppfull.as<int>(), yN, s->C, s->Pq, mu,
                                                                       sd, s->xb.as<bf16>(), nullptr);
        S_CUDA(s, cudaGetLastError());
        ctx->launches++;
        if ((rc = forward(s, 1))) return rc;
        if (dst) {
            cv_write<<<blocks_for(s->Pq * s->C), 256, 0, ctx->stream>>>(
                s->out.as<float>(), s->out_ref.as<float>(), s->Eref.as<double>(), s->ppfull.as<int>(), yN, s->C,
                s->Pq, so, dst);
            S_CUDA(s, cudaGetLastError());
            ctx->launches++;
        }
        return RTBTE_OK;
    }
    if (!s->smem_set) {
        S_CUDA(s, allow_max_dynamic_smem((const void *)infer_conv<0>));
        S_CUDA(s, allow_max_dynamic_smem((const void *)infer_conv<1>));
        S_CUDA(s, allow_max_dynamic_smem((const void *)infer_conv<2>));
        s->smem_set = true;
    }
    InferArgs a{};
    a.y = y;
    a.pp_full = s->ppfull.as<int>();
    a.yN = yN;
    a.Pq = s->Pq;
    a.mu = mu;
    a.sd = sd;
    a.so = so;
    a.C = s->C;
    a.ny = s->ny;
    a.nx = s->nx;
    const bf16 *wt = s->wbt.as<bf16>();
    const int grid = (int)((s->Pq + kIM - 1) / kIM);
    bf16 *bufs[2] = {s->a0.as<bf16>(), s->a1.as<bf16>()};
    for (int l = 0; l < kLayers; ++l) {
        a.KP = s->kpad[l];
        a.Wt = wt + s->off_t[l];
        a.bias = s->w.as<float>() + s->off_b[l];
        a.act_in = l > 0 ? bufs[(l - 1) & 1] : nullptr;
        a.act_out = bufs[l & 1];
        if (l == 0) {
            infer_conv<0><<<grid, kIThreads, infer_smem(a.KP, 0), ctx->stream>>>(a);
        } else if (l < kLayers - 1) {
            infer_conv<1><<<grid, kIThreads, infer_smem(a.KP, 1), ctx->stream>>>(a);
        } else {
            a.M1t = wt + s->off_t[kLayers];
            a.c1 = s->w.as<float>() + s->off_c1;
            a.M2 = s->wb.as<bf16>() + s->off_M2;
            a.c2 = s->w.as<float>() + s->off_c2;
            a.out = s->out.as<float>();
            a.out_ref = s->out_ref.as<float>();
            a.Eref = s->Eref.as<double>();
            a.dst = dst;
            infer_conv<2><<<grid, kIThreads, infer_smem(a.KP, 2), ctx->stream>>>(a);
        }
        S_CUDA(s, cudaGetLastError());
    }
    ctx->launches += kLayers;
    return RTBTE_OK;
}

int ensure_ref(rtbte_surrogate *s) {
    if (s->Eref.p) return RTBTE_OK;
    int rc;
    if ((rc = salloc(s, s->Eref, sizeof(double) * s->Pq * s->C)) ||
        (rc = salloc(s, s->out_ref, sizeof(float) * s->Pq * s->C)) || (rc = salloc(s, s->normp, sizeof(double) * 2 * 512)))
        return rc;
    S_CUDA(s, cudaMemsetAsync(s->Eref.p, 0, sizeof(double) * s->Pq * s->C, s->ctx->stream));
    S_CUDA(s, cudaMemsetAsync(s->out_ref.p, 0, sizeof(float) * s->Pq * s->C, s->ctx->stream));
    return RTBTE_OK;
}

}  // namespace

namespace rtbte {

int sur_value(rtbte_ctx *ctx, const double *y, double *dst) {
    rtbte_surrogate *s = ctx->sur;
    if (!s || !s->has_ref) return fail(ctx, RTBTE_E_STATE, "surrogate has no exact reference");
    int rc;
    if ((rc = infer(s, y, dst))) return fail(ctx, rc, s->err);
    return RTBTE_OK;
}

int sur_judge(rtbte_ctx *ctx, const double *y, const double *exact, double *relerr) {
    rtbte_surrogate *s = ctx->sur;
    int rc;
    if (!s) return fail(ctx, RTBTE_E_STATE, "no surrogate attached");
    if ((rc = ensure_ref(s)) || (rc = infer(s, y, nullptr))) return fail(ctx, rc, s->err);
    const InstHost &I = ctx->inst[s->inst];
    const long long n = s->Pq * s->C;
    const int nb = (int)std::min<long long>(512, (n + 255) / 256);
    judge_cv<<<nb, 256, 0, ctx->stream>>>(s->out.as<float>(), s->out_ref.as<float>(), s->Eref.as<double>(), exact,
                                          s->ppfull.as<int>(), I.y_off + I.d.n_c, s->C, s->Pq,
                                          s->stats.as<float>() + 32, s->normp.as<double>());
    RT_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    *relerr = -1.0;
    if (s->has_ref) {
        std::vector<double> part(2 * nb);
        RT_CUDA(ctx, cudaMemcpyAsync(part.data(), s->normp.p, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost,
                                     ctx->stream));
        RT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        double d2 = 0, e2 = 0;
        for (int b = 0; b < nb; ++b) {
            d2 += part[2 * b];
            e2 += part[2 * b + 1];
        }
        *relerr = e2 > 0 ? sqrt(d2 / e2) : (d2 > 0 ? INFINITY : 0.0);
    }
    s->has_ref = true;
    return RTBTE_OK;
}

void sur_orphan(rtbte_ctx *ctx) {
    for (rtbte_surrogate *s : ctx->surs) s->ctx = nullptr;
    ctx->surs.clear();
    ctx->sur = nullptr;
}

void sur_reset(rtbte_ctx *ctx) {
    if (ctx->sur) ctx->sur->has_ref = false;
}

}  // namespace rtbte

extern "C" {

int rtbte_set_surrogate(rtbte_ctx *ctx, rtbte_surrogate *s, int judge_period, double judge_tol) {
    if (!ctx) return RTBTE_E_INVALID_ARG;
    if (!s) {
        ctx->sur = nullptr;
        return RTBTE_OK;
    }
    if (s->ctx != ctx || judge_period < 1 || !(judge_tol > 0)) return fail(ctx, RTBTE_E_INVALID_ARG, "bad surrogate");
    if (ctx->inst.size() != 1 || s->inst != 0)
        return fail(ctx, RTBTE_E_UNSUPPORTED, "surrogate MRI needs a single-instance context");
    if (!s->stats_set) return fail(ctx, RTBTE_E_STATE, "surrogate not trained");
    ctx->sur = s;
    ctx->sur_period = judge_period;
    ctx->sur_tol = judge_tol;
    s->has_ref = false;
    return RTBTE_OK;
}

int rtbte_surrogate_create(rtbte_ctx *ctx, int inst, int width, int capacity, uint64_t seed, rtbte_surrogate **out) {
    if (!ctx || !out || inst < 0 || inst >= (int)ctx->inst.size() || width < 8 || width > 256 || width % 8 ||
        capacity < 1)
        return RTBTE_E_INVALID_ARG;
    InstHost &I = ctx->inst[inst];
    if (I.M == 0 || I.d.dim != 2 || I.d.nmodes > 16) return RTBTE_E_UNSUPPORTED;
    rtbte_surrogate *s = new rtbte_surrogate();
    s->ctx = ctx;
    s->inst = inst;
    s->C = I.d.nmodes;
    s->width = width;
    s->nx = I.nqs[0];
    s->ny = I.nqs[1];
    s->Pq = I.N_qs;
    s->capacity = capacity;
    s->rng.seed(seed);
    const int cin[kLayers] = {s->C, width, width, width};
    long long off = 0;
    for (int l = 0; l < kLayers; ++l) {
        s->cin[l] = cin[l];
        s->kpad[l] = (9 * cin[l] + kBK - 1) / kBK * kBK;
        s->off_W[l] = off;
        off += (long long)s->kpad[l] * width;
        s->off_b[l] = off;
        off += width;
    }
    s->off_M1 = off;
    off += (long long)width * width;
    s->off_c1 = off;
    off += width;
    s->off_M2 = off;
    off += (long long)width * s->C;
    s->off_c2 = off;
    off += s->C;
    s->nparam = off;
    int rc;
    auto bail = [&](int c) {
        rtbte_surrogate_destroy(s);
        return c;
    };
    if ((rc = salloc(s, s->w, sizeof(float) * off)) || (rc = salloc(s, s->wb, sizeof(bf16) * off)) ||
        (rc = salloc(s, s->g, sizeof(float) * off)) || (rc = salloc(s, s->m, sizeof(float) * off)) ||
        (rc = salloc(s, s->v, sizeof(float) * off)) || (rc = salloc(s, s->stats, sizeof(float) * 48)) ||
        (rc = salloc(s, s->ppfull, sizeof(int) * I.M)) || (rc = salloc(s, s->ydot, sizeof(double) * ctx->n_y)) ||
        (rc = salloc(s, s->Ns, sizeof(float) * (long long)capacity * s->Pq * s->C)) ||
        (rc = salloc(s, s->Is, sizeof(float) * (long long)capacity * s->Pq * s->C)))
        return bail(rc);
    // pp_full of the instance in [c][q_s] order, as instance-local phonon index (row offset n_c added by callers)
    std::vector<int> pf(I.M);
    for (long long a = 0; a < I.M; ++a) pf[a] = I.pp_full[a];
    if (cudaMemcpy(s->ppfull.p, pf.data(), sizeof(int) * I.M, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(RTBTE_E_CUDA);
    cudaMemset(s->m.p, 0, sizeof(float) * off);
    cudaMemset(s->v.p, 0, sizeof(float) * off);
    // initial weights: N(0, 1/fan_in), last layer scaled by 0.1, biases 0
    std::vector<float> w(off, 0.f);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int l = 0; l < kLayers; ++l) {
        const float sc = 1.f / sqrtf(9.f * cin[l]);
        for (long long r = 0; r < 9LL * cin[l]; ++r)
            for (int c = 0; c < width; ++c) w[s->off_W[l] + r * width + c] = sc * nd(s->rng);
    }
    for (long long i = 0; i < (long long)width * width; ++i) w[s->off_M1 + i] = nd(s->rng) / sqrtf((float)width);
    for (long long i = 0; i < (long long)width * s->C; ++i) w[s->off_M2 + i] = 0.1f * nd(s->rng) / sqrtf((float)width);
    if (cudaMemcpy(s->w.p, w.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(RTBTE_E_CUDA);
    to_bf16<<<blocks_for(off), 256, 0, ctx->stream>>>(s->w.as<float>(), off, s->wb.as<bf16>());
    // tensor-core GEMMs (tcgen05) when the device has them and TMA maps can be made
    {
        int cc = 0;
        cudaDeviceGetAttribute(&cc, cudaDevAttrComputeCapabilityMajor, ctx->device);
        s->engine = (cc >= 10 && encode_tiled()) ? 0 : 1;
        long long t = 0;
        for (int l = 0; l < kLayers; ++l) {
            s->off_tt[l] = t;
            t += (long long)s->kpad[l] * width;
        }
        s->off_tt[kLayers] = t;
        t += (long long)width * width;
        s->off_tt[kLayers + 1] = t;
        t += (long long)width * s->C;
        if ((rc = salloc(s, s->wtt, sizeof(bf16) * t)) || (rc = salloc(s, s->tcerr, sizeof(int)))) return bail(rc);
        cudaMemset(s->tcerr.p, 0, sizeof(int));
        if ((rc = refresh_training_layout(s))) return bail(rc);
    }
    s->fused = width == kIW;
    if (s->fused) {
        long long t = 0;
        for (int l = 0; l < kLayers; ++l) {
            s->off_t[l] = t;
            t += (long long)s->kpad[l] * kIW;
        }
        s->off_t[kLayers] = t;
        t += (long long)kIW * kIW;
        if ((rc = salloc(s, s->wbt, sizeof(bf16) * t)) || (rc = salloc(s, s->a0, sizeof(bf16) * s->Pq * kIW)) ||
            (rc = salloc(s, s->a1, sizeof(bf16) * s->Pq * kIW)) || (rc = refresh_inference(s)))
            return bail(rc);
    }
    for (int c = 0; c < s->C; ++c) {
        s->mu[c] = 0.f;
        s->sd[c] = 1.f;
        s->so[c] = 1.f;
    }
    if ((rc = upload_stats(s))) return bail(rc);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return bail(RTBTE_E_CUDA);
    ctx->surs.push_back(s);
    *out = s;
    return RTBTE_OK;
}

int rtbte_surrogate_collect(rtbte_surrogate *s, const double *y, int trajectory) {
    if (!s || !y) return RTBTE_E_INVALID_ARG;
    if (!s->ctx) return sfail(s, RTBTE_E_STATE, "context destroyed");
    if (s->count >= s->capacity) return sfail(s, RTBTE_E_INVALID_ARG, "pair buffer full");
    rtbte_ctx *ctx = s->ctx;
    int rc = rtbte_rhs(ctx, 0.0, y, s->ydot.as<double>(), RTBTE_SLOW);
    if (rc) return sfail(s, rc, rtbte_last_error(ctx));
    const InstHost &I = ctx->inst[s->inst];
    const long long per = s->Pq * s->C;
    gather_pair<<<blocks_for(per), 256, 0, ctx->stream>>>(y, s->ydot.as<double>(), s->ppfull.as<int>(),
                                                          I.y_off + I.d.n_c, s->C, s->Pq,
                                                          s->Ns.as<float>() + (long long)s->count * per,
                                                          s->Is.as<float>() + (long long)s->count * per);
    S_CUDA(s, cudaGetLastError());
    ctx->launches++;
    s->count++;
    s->traj.push_back(trajectory);
    return RTBTE_OK;
}

int rtbte_surrogate_train(rtbte_surrogate *s, int steps, int batch, int horizon, float lr, float *loss_out) {
    if (!s || steps < 0 || batch < 1 || horizon < 0) return RTBTE_E_INVALID_ARG;
    if (!s->ctx) return sfail(s, RTBTE_E_STATE, "context destroyed");
    if (s->count < 1) return sfail(s, RTBTE_E_STATE, "no collected pairs");
    rtbte_ctx *ctx = s->ctx;
    int rc;
    const int nsamp = horizon > 0 ? 2 * batch : batch;
    if ((rc = ensure_batch(s, nsamp))) return rc;
    const long long per = s->Pq * s->C;
    if (!s->stats_set) {  // per-channel normalisation from the collected pairs (host, FP64)
        std::vector<float> N((size_t)s->count * per), I((size_t)s->count * per);
        S_CUDA(s, cudaMemcpy(N.data(), s->Ns.p, sizeof(float) * N.size(), cudaMemcpyDeviceToHost));
        S_CUDA(s, cudaMemcpy(I.data(), s->Is.p, sizeof(float) * I.size(), cudaMemcpyDeviceToHost));
        for (int c = 0; c < s->C; ++c) {
            double a = 0, a2 = 0, b2 = 0;
            long long n = 0;
            for (size_t i = c; i < N.size(); i += s->C) {
                a += N[i];
                a2 += (double)N[i] * N[i];
                b2 += (double)I[i] * I[i];
                ++n;
            }
            const double mean = a / n, var = a2 / n - mean * mean;
            s->mu[c] = (float)mean;
            s->sd[c] = (float)std::max(sqrt(std::max(var, 0.0)), 1e-6);
            s->so[c] = (float)std::max(sqrt(b2 / n), 1e-30);
        }
        if ((rc = upload_stats(s))) return rc;
        s->stats_set = true;
    }
    // training units: single samples, or (later, earlier) pairs of one trajectory at most
    // `horizon` collections apart
    std::vector<std::pair<int, int>> units;
    if (horizon == 0) {
        for (int i = 0; i < s->count; ++i) units.emplace_back(i, -1);
    } else {
        for (int j = 0; j < s->count; ++j)
            for (int i = std::max(0, j - horizon); i < j; ++i)
                if (s->traj[i] == s->traj[j]) units.emplace_back(j, i);
        if (units.empty()) return sfail(s, RTBTE_E_STATE, "no pairs of one trajectory within the horizon");
    }
    const float *mu = s->stats.as<float>(), *sd = mu + 16, *so = mu + 32;
    std::vector<int> perm(units.size());
    for (size_t i = 0; i < perm.size(); ++i) perm[i] = (int)i;
    size_t pos = perm.size();
    std::vector<int> bidx(nsamp);
    float last = 0.f;
    for (int it = 0; it < steps; ++it) {
        for (int b = 0; b < batch; ++b) {
            if (pos >= perm.size()) {
                std::shuffle(perm.begin(), perm.end(), s->rng);
                pos = 0;
            }
            const auto &u = units[perm[pos++]];
            bidx[b] = u.first;
            if (horizon > 0) bidx[batch + b] = u.second;
        }
        S_CUDA(s, cudaMemcpyAsync(s->idx.p, bidx.data(), sizeof(int) * nsamp, cudaMemcpyHostToDevice, ctx->stream));
        gather_batch<<<blocks_for(nsamp * per), 256, 0, ctx->stream>>>(s->Ns.as<float>(), s->Is.as<float>(),
                                                                      s->idx.as<int>(), nsamp, s->C, s->Pq, mu, sd, so,
                                                                      s->xb.as<bf16>(), s->t.as<float>());
        S_CUDA(s, cudaGetLastError());
        ctx->launches++;
        if ((rc = loss_grad(s, nsamp, it == steps - 1 ? &last : nullptr, horizon > 0))) return rc;
        s->adam_t++;
        const float b1 = 0.9f, b2 = 0.999f;
        adam<<<blocks_for(s->nparam), 256, 0, ctx->stream>>>(
            s->w.as<float>(), s->g.as<float>(), s->m.as<float>(), s->v.as<float>(), s->nparam, lr, b1, b2, 1e-8f,
            1.f - powf(b1, (float)s->adam_t), 1.f - powf(b2, (float)s->adam_t), s->wb.as<bf16>());
        S_CUDA(s, cudaGetLastError());
        ctx->launches++;
        if ((rc = refresh_training_layout(s))) return rc;
    }
    if ((rc = refresh_inference(s))) return rc;
    S_CUDA(s, cudaStreamSynchronize(ctx->stream));
    if ((rc = check_tc(s))) return rc;
    if (loss_out) *loss_out = last;
    return RTBTE_OK;
}

int rtbte_surrogate_predict(rtbte_surrogate *s, const double *y, double *out) {
    if (!s || !y || !out) return RTBTE_E_INVALID_ARG;
    if (!s->ctx) return sfail(s, RTBTE_E_STATE, "context destroyed");
    rtbte_ctx *ctx = s->ctx;
    int rc;
    if ((rc = infer(s, y, nullptr))) return rc;
    const InstHost &I = ctx->inst[s->inst];
    S_CUDA(s, cudaMemsetAsync(out, 0, sizeof(double) * ctx->n_y, ctx->stream));
    scatter_output<<<blocks_for(s->Pq * s->C), 256, 0, ctx->stream>>>(
        s->out.as<float>(), s->ppfull.as<int>(), I.y_off + I.d.n_c, s->C, s->Pq, s->stats.as<float>() + 32, out);
    S_CUDA(s, cudaGetLastError());
    ctx->launches++;
    return RTBTE_OK;
}

int64_t rtbte_surrogate_num_params(const rtbte_surrogate *s) {
    if (!s) return 0;
    long long n = 0;
    for (int l = 0; l < kLayers; ++l) n += 9LL * s->cin[l] * s->width + s->width;
    return n + (long long)s->width * s->width + s->width + (long long)s->width * s->C + s->C;
}

int rtbte_surrogate_get_params(rtbte_surrogate *s, float *host) {
    if (!s || !host) return RTBTE_E_INVALID_ARG;
    if (!s->ctx) return sfail(s, RTBTE_E_STATE, "context destroyed");
    return params_io(s, host, false);
}

int rtbte_surrogate_set_params(rtbte_surrogate *s, const float *host) {
    if (!s || !host) return RTBTE_E_INVALID_ARG;
    if (!s->ctx) return sfail(s, RTBTE_E_STATE, "context destroyed");
    int rc = params_io(s, const_cast<float *>(host), true);
    if (rc || (rc = refresh_inference(s)) || (rc = refresh_training_layout(s))) return rc;
    S_CUDA(s, cudaStreamSynchronize(s->ctx->stream));
    return RTBTE_OK;
}

int rtbte_surrogate_set_gemm(rtbte_surrogate *s, int engine) {
    if (!s || engine < 0 || engine > 1) return RTBTE_E_INVALID_ARG;
    if (!s->ctx) return sfail(s, RTBTE_E_STATE, "context destroyed");
    if (engine == 0) {
        int cc = 0;
        cudaDeviceGetAttribute(&cc, cudaDevAttrComputeCapabilityMajor, s->ctx->device);
        if (cc < 10 || !encode_tiled()) return sfail(s, RTBTE_E_UNSUPPORTED, "no tcgen05 tensor cores or TMA maps");
    }
    s->engine = engine;
    int rc;
    if ((rc = refresh_training_layout(s))) return rc;
    S_CUDA(s, cudaStreamSynchronize(s->ctx->stream));
    return RTBTE_OK;
}

int rtbte_surrogate_loss_grad(rtbte_surrogate *s, const float *x, const float *t, int B, float *loss, float *grad,
                              float *out) {
    if (!s || !x || !t || B < 1 || !loss) return RTBTE_E_INVALID_ARG;
    if (!s->ctx) return sfail(s, RTBTE_E_STATE, "context destroyed");
    int rc;
    if ((rc = ensure_batch(s, B))) return rc;
    const long long n = (long long)B * s->Pq * s->C;
    std::vector<bf16> xb(n);
    for (long long i = 0; i < n; ++i) xb[i] = __float2bfloat16(x[i]);
    S_CUDA(s, cudaMemcpy(s->xb.p, xb.data(), sizeof(bf16) * n, cudaMemcpyHostToDevice));
    S_CUDA(s, cudaMemcpy(s->t.p, t, sizeof(float) * n, cudaMemcpyHostToDevice));
    if ((rc = loss_grad(s, B, loss)) || (rc = check_tc(s))) return rc;
    if (out) S_CUDA(s, cudaMemcpy(out, s->out.p, sizeof(float) * n, cudaMemcpyDeviceToHost));
    if (grad) {
        // gradients in the logical layout
        DevBuf saved = s->w;
        s->w = s->g;
        rc = params_io(s, grad, false);
        s->w = saved;
        saved.p = nullptr;
        if (rc) return rc;
    }
    return RTBTE_OK;
}

void rtbte_surrogate_stats(const rtbte_surrogate *s, float *mu, float *sd, float *so, int *count) {
    if (!s) return;
    for (int c = 0; c < s->C; ++c) {
        if (mu) mu[c] = s->mu[c];
        if (sd) sd[c] = s->sd[c];
        if (so) so[c] = s->so[c];
    }
    if (count) *count = s->count;
}

void rtbte_surrogate_destroy(rtbte_surrogate *s) {
    if (!s) return;
    if (s->ctx) {
        cudaStreamSynchronize(s->ctx->stream);
        if (s->ctx->sur == s) s->ctx->sur = nullptr;
        auto &v = s->ctx->surs;
        v.erase(std::remove(v.begin(), v.end(), s), v.end());
    }
    DevBuf *bufs[] = {&s->w,  &s->wb,  &s->g,     &s->m,    &s->v,     &s->stats, &s->ppfull, &s->Ns,
                      &s->Is, &s->idx, &s->xb,    &s->t,    &s->out,   &s->gout,  &s->goutb,  &s->ga,
                      &s->gz, &s->gzb, &s->gcol,  &s->split, &s->lossp, &s->ydot, &s->Eref,   &s->out_ref,
                      &s->normp, &s->wbt, &s->a0,  &s->a1, &s->wtt, &s->tcerr};
    for (DevBuf *b : bufs) b->release();
    for (int l = 0; l < kLayers; ++l) s->cols[l].release();
    for (int l = 0; l <= kLayers; ++l) {
        s->acts[l].release();
        s->actb[l].release();
    }
    delete s;
}

}  // extern "C"
