// noalloc.cu -- an e-ph RHS entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: programs whose device memory is owned entirely by
// another allocator or by an arena reserved at start-up (a serving runtime, a host
// application that budgets every byte of the GPU), and latency-critical loops where an
// allocation's implicit device synchronisation is not acceptable.  rtbte_eph_rhs_noalloc
// serves them: the caller passes every input and output as device pointers, and the only
// working memory (single-precision copies of the populations and one compensated partial sum
// per list segment) lives in the file-scope array below, which every device that loads this
// library holds until the process exits.
//
// The arithmetic is that of the collision kernel in rhs.cu restricted to the electron rows
// of the e-ph integral: FP32 gathers and products, per-lane two-sum accumulation, a
// compensated warp reduction per segment, and the segment partials added in a fixed order
// in FP64, so the result matches rtbte_rhs(RTBTE_EPH) to FP32 rounding.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "rtbte.h"

namespace {

constexpr long long kScratchFloats = RTBTE_NOALLOC_SCRATCH_BYTES / 4;
constexpr int kMaxDevices = 64;
constexpr unsigned kFull = 0xffffffffu;

// The scratch array shared by every call on a device.
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

std::mutex g_mu;
float *g_addr[kMaxDevices] = {};

__global__ void na_prep(const double *y, float *f, float *N, int n_c, long long n_ph) {
    const long long n = (long long)n_c + n_ph;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (i < n_c) f[i] = (float)y[i];
        else N[i - n_c] = (float)y[i];
    }
}

__device__ __forceinline__ void na_two_sum(float &s, float &c, float x) {
    float t = s + x;
    float bp = t - s;
    float e = (s - (t - bp)) + (x - bp);
    s = t;
    c += e;
}

// One warp per segment g = (nu*n_c + d)*2 + proc of the e-ph list; writes partial[g].
__global__ void na_segments(const int64_t *off, const int32_t *src, const int32_t *ph, const double *W,
                            const float *f, const float *N, float2 *partial, int n_c, long long nseg) {
    const int lane = threadIdx.x & 31;
    for (long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; g < nseg;
         g += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int d = (int)((g >> 1) % n_c);
        const int proc = (int)(g & 1);
        const float fd = f[d];
        float acc = 0.f, cmp = 0.f;
        for (long long e = off[g] + lane; e < off[g + 1]; e += 32) {
            const float fs = f[src[e]];
            const float n = N[ph[e]];
            const float F = proc ? n * (fd - fs) - fs * (1.f - fd) : fd * (1.f - fs) + n * (fd - fs);
            na_two_sum(acc, cmp, (float)W[e] * F);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            float s2 = __shfl_xor_sync(kFull, acc, o), c2 = __shfl_xor_sync(kFull, cmp, o);
            float t = acc + s2, bp = t - acc, e = (acc - (t - bp)) + (s2 - bp);
            acc = t;
            cmp = (cmp + c2) + e;
        }
        if (lane == 0) partial[g] = make_float2(acc, cmp);
    }
}

__global__ void na_rows(const float2 *partial, double *ydot, int n_c, int nmodes) {
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < n_c; d += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int nu = 0; nu < nmodes; ++nu)
            for (int proc = 0; proc < 2; ++proc) {
                const float2 p = partial[((long long)nu * n_c + d) * 2 + proc];
                acc += (double)p.x + (double)p.y;
            }
        ydot[d] = -acc;
    }
}

}  // namespace

extern "C" int rtbte_eph_rhs_noalloc(int32_t n_c, int64_t n_ph, int32_t nmodes, const int64_t *off,
                                     const int32_t *src, const int32_t *ph, const double *W, const double *y,
                                     double *ydot, void *stream) {
    if (n_c < 1 || nmodes < 1 || n_ph < nmodes) return RTBTE_E_INVALID_ARG;
    const long long nseg = 2LL * nmodes * n_c;
    // floats: f copy (n_c, rounded to 4), N copy (n_ph, rounded to 4), two per segment partial
    const long long fpad = (n_c + 3) / 4 * 4, npad = (n_ph + 3) / 4 * 4;
    if (fpad + npad + 2 * nseg > kScratchFloats) return RTBTE_E_UNSUPPORTED;
    if (!off || !src || !ph || !W || !y || !ydot) return RTBTE_E_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return RTBTE_E_CUDA;
    }
    float *base;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return RTBTE_E_CUDA;
            }
            g_addr[dev] = reinterpret_cast<float *>(p);
        }
        base = g_addr[dev];
    }
    float *f = base, *N = base + fpad;
    float2 *partial = reinterpret_cast<float2 *>(base + fpad + npad);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return RTBTE_E_CUDA;
    }
    const long long n = n_c + n_ph;
    na_prep<<<(unsigned)std::min<long long>((n + 255) / 256, 8LL * sms), 256, 0, s>>>(y, f, N, n_c, n_ph);
    na_segments<<<(unsigned)std::min<long long>((nseg * 32 + 255) / 256, 32LL * sms), 256, 0, s>>>(
        off, src, ph, W, f, N, partial, n_c, nseg);
    na_rows<<<(unsigned)std::min<long long>((n_c + 255) / 256, 8LL * sms), 256, 0, s>>>(partial, ydot, n_c, nmodes);
    if (cudaGetLastError() != cudaSuccess) return RTBTE_E_CUDA;
    return RTBTE_OK;
}
