// nfft.cu -- the nonlinear FFT of Sec. 3 (radix-2 with the operator of Eq. 6 in
// every butterfly), decimation in time (the recursion of Sec. 3) or, with
// NDFT_F_NFFT_DIF, decimation in frequency; and the cross-ambiguity surface of
// Eq. 12a evaluated through it.  The kernels are the op/direction templates of
// fft_core.cuh; N > 65536 (plain DIT transforms only) runs one launch per stage
// over global memory.
#include "fft_core.cuh"

namespace ndft {

namespace {

// ---- N > 65536 (plain NFFT only): bit reversal, then one launch per stage ----------
__device__ __forceinline__ void butterfly(float2 *a, int64_t i0, int64_t i1, float2 w) {
    const float2 E = a[i0];
    const float2 t = cox_f32(w, a[i1]);
    a[i0] = make_float2(__fadd_rn(E.x, t.x), __fadd_rn(E.y, t.y));
    a[i1] = make_float2(__fsub_rn(E.x, t.x), __fsub_rn(E.y, t.y));
}

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

size_t nfft_ws_bytes(const ndft_desc &d, int64_t *chunk) {
    *chunk = 0;
    const int64_t N = d.n;
    if (d.prec != NDFT_PREC_FP32 || N < 8192 || N > 65536 || (N & (N - 1))) return 0;
    int64_t want = d.max_batch;
    if ((d.form == NDFT_FORM_NFFT || d.form == NDFT_FORM_FFT) && d.max_lags > want) want = d.max_lags;
    if (want <= 0) return 0;
    int64_t ch = (int64_t)(kNfftChunkBytes / (N * (int64_t)sizeof(float2)));
    if (ch < 1) ch = 1;
    if (ch > want) ch = want;
    *chunk = ch;
    return (size_t)ch * N * sizeof(float2);
}

cudaError_t launch_nfft(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s, int *launches) {
    const int N = p.d.n;
    if (batch == 0) return cudaSuccess;
    const bool dif = p.d.flags & NDFT_F_NFFT_DIF;
    if (N <= 65536) {
        return dif ? fft_vectors<OpNL, true>(p, x, X, batch, s, launches)
                   : fft_vectors<OpNL, false>(p, x, X, batch, s, launches);
    }
    if (dif) return cudaErrorInvalidValue;
    const int logN = log2i(N);
    const float2 *xi = static_cast<const float2 *>(x);
    float2 *Xo = static_cast<float2 *>(X);
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

cudaError_t launch_nfft_bins(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s,
                             int *launches) {
    return (p.d.flags & NDFT_F_NFFT_DIF) ? fft_bins<OpNL, true>(p, x, X, batch, s, launches)
                                         : fft_bins<OpNL, false>(p, x, X, batch, s, launches);
}

cudaError_t launch_nfft_caf(const Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags, void *A,
                            cudaStream_t s, int *launches) {
    return (p.d.flags & NDFT_F_NFFT_DIF) ? fft_caf<OpNL, true>(p, s_surv, s_ref, lag0, nlags, A, s, launches)
                                         : fft_caf<OpNL, false>(p, s_surv, s_ref, lag0, nlags, A, s, launches);
}

}  // namespace ndft
