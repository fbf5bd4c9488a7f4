// nfft.cu -- the nonlinear FFT of Sec. 3: radix-2 decimation in time with the
// twiddle product of every butterfly replaced by the operator of Eq. 6.
//
// With the input in bit-reversed order, stage s (span L = 2^s) turns each pair
// of L/2-point NFFTs E, O into the L-point NFFT
//     t = W_L^k (x) O[k],   X[k] = E[k] + t,   X[k + L/2] = E[k] - t,
// W_L^k = W_N^(k N / L) read from the plan's fp32 table.  Every real (x) is
// rounded once and each add/subtract once, in this order, so the output is
// reproducible bit for bit.  Radix-4/8 regrouping would change the result
// (W1 (x) (W2 (x) v) != (W1 W2) (x) v), so only data movement is optimised:
// up to N = 16384 a vector stays in shared memory for all stages.
#include "internal.cuh"

namespace ndft {

namespace {

__device__ __forceinline__ uint32_t bitrev(uint32_t v, int bits) { return __brev(v) >> (32 - bits); }

__device__ __forceinline__ void butterfly(float2 *a, int64_t i0, int64_t i1, float2 w) {
    const float2 E = a[i0];
    const float2 t = cox_f32(w, a[i1]);
    a[i0] = make_float2(__fadd_rn(E.x, t.x), __fadd_rn(E.y, t.y));
    a[i1] = make_float2(__fsub_rn(E.x, t.x), __fsub_rn(E.y, t.y));
}

// V vectors of N points per block, all stages in shared memory.
__global__ void k_nfft_smem(const float2 *__restrict__ x, float2 *__restrict__ X, const float2 *__restrict__ tw,
                            int N, int logN, int V, int64_t batch) {
    extern __shared__ __align__(16) float2 sa[];
    const int64_t v0 = (int64_t)blockIdx.x * V;
    const int nv = (int)((batch - v0) < V ? (batch - v0) : V);
    const int total = nv * N;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int v = e / N, n = e - v * N;
        sa[v * N + bitrev(n, logN)] = x[(v0 + v) * N + n];
    }
    __syncthreads();
    const int nb = nv * (N / 2);
    for (int s = 1; s <= logN; ++s) {
        const int half = 1 << (s - 1);
        const int tstep = N >> s;  // N / L
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int v = b / (N / 2), bb = b - v * (N / 2);
            const int g = bb >> (s - 1), k = bb & (half - 1);
            const int i0 = v * N + (g << s) + k;
            butterfly(sa, i0, i0 + half, __ldg(&tw[k * tstep]));
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < total; e += blockDim.x) X[v0 * N + e] = sa[e];
}

// Large N: bit-reversal permutation (in place or out of place), then one
// launch per stage over global memory.
__global__ void k_bitrev(const float2 *__restrict__ x, float2 *__restrict__ X, int N, int logN, int64_t batch,
                         bool inplace) {
    const int64_t total = batch * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / N;
        const uint32_t n = (uint32_t)(e - v * N);
        const uint32_t r = bitrev(n, logN);
        if (inplace) {
            if (n < r) {
                const float2 a = X[v * N + n];
                X[v * N + n] = X[v * N + r];
                X[v * N + r] = a;
            }
        } else {
            X[v * N + r] = x[v * N + n];
        }
    }
}

__global__ void k_stage(float2 *__restrict__ X, const float2 *__restrict__ tw, int N, int s, int64_t batch) {
    const int half = 1 << (s - 1);
    const int tstep = N >> s;
    const int64_t total = batch * (N / 2);
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < total;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = b / (N / 2);
        const int bb = (int)(b - v * (N / 2));
        const int g = bb >> (s - 1), k = bb & (half - 1);
        const int64_t i0 = v * N + ((int64_t)g << s) + k;
        butterfly(X, i0, i0 + half, __ldg(&tw[(int64_t)k * tstep]));
    }
}

}  // namespace

cudaError_t launch_nfft(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s, int *launches) {
    const int N = p.d.n;
    int logN = 0;
    while ((1 << logN) < N) ++logN;
    if (batch == 0) return cudaSuccess;
    const float2 *xi = static_cast<const float2 *>(x);
    float2 *Xo = static_cast<float2 *>(X);
    if (N <= 16384) {
        const int V = N >= 2048 ? 1 : 2048 / N;
        const size_t smem = (size_t)V * N * sizeof(float2);
        cudaError_t e = cudaFuncSetAttribute(k_nfft_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int threads = (V * N / 2) >= 512 ? 512 : (V * N / 2 >= 32 ? V * N / 2 : 32);
        const int64_t blocks = (batch + V - 1) / V;
        if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
        timer_begin(p, s);
        k_nfft_smem<<<(unsigned)blocks, threads, smem, s>>>(xi, Xo, p.tw32, N, logN, V, batch);
        timer_end(p, s);
        *launches += 1;
        return cudaGetLastError();
    }
    const int threads = 256;
    const int blocks = p.sm_count * 8;
    k_bitrev<<<blocks, threads, 0, s>>>(xi, Xo, N, logN, batch, xi == Xo);
    *launches += 1;
    for (int st = 1; st <= logN; ++st) {
        k_stage<<<blocks, threads, 0, s>>>(Xo, p.tw32, N, st, batch);
        *launches += 1;
    }
    return cudaGetLastError();
}

}  // namespace ndft
