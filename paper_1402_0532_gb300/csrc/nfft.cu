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

// 8 <= N <= 4096: each thread keeps 8 points in registers and runs up to 3
// radix-2 stages on them between shared-memory exchanges.  In the pass that
// starts at stage bit B0 the thread's points differ in the 3 index bits
// [W, W + 3), W = min(B0, logN - 3), so every stage whose butterfly distance
// 2^b lies in that window pairs two of its own points; stages already done in
// earlier passes are skipped.  The butterflies and their order within each
// stage are those of the stage loop above, so results are identical bit for
// bit.
//
// Data movement: the first pass reads its points straight from global memory
// (thread t of a vector takes the group whose bit-reversed positions are
// 8 rev(t) + j, i.e. natural indices t + rev3(j) N/8: coalesced), and the last
// pass writes straight to global memory (positions t + j N/8, natural order).
// Only the passes in between exchange through shared memory, under an XOR
// swizzle of the low 4 index bits that keeps every exchange free of bank
// conflicts.  Twiddles sit in shared memory as one table per stage, indexed by
// k, so a warp reads consecutive entries; each entry is the twiddle in
// "ready" form (|Re|, |Im|, sgn Re, sgn Im).
__device__ __forceinline__ int swz(int p) { return p ^ ((p >> 4) & 15) ^ ((p >> 8) & 15) ^ ((p >> 3) & 8); }

// sgn(v) as 1.0f, 0.0f or -1.0f.
__device__ __forceinline__ float sgnf(float v) {
    float g, l;
    asm("set.gt.f32.f32 %0, %1, 0f00000000;" : "=f"(g) : "f"(v));
    asm("set.lt.f32.f32 %0, %1, 0f00000000;" : "=f"(l) : "f"(v));
    return __fsub_rn(g, l);
}

// Eq. 6 with the twiddle in ready form.  Each real a (x) b = sgn(a) sgn(b)
// (|a| + |b|) is formed as fma(sgn a, fma(sgn b, |a|, b), +0): the inner fma
// rounds sgn(b)(|a| + |b|) once (round to nearest is symmetric), the outer one
// scales it exactly by sgn a, and the +0 addend turns every zero product into
// +0, as the definition's 0 for a zero operand.  Same bits as cox_f32.
__device__ __forceinline__ float2 cox_ready(float4 w, float2 o) {
    const float sx = sgnf(o.x), sy = sgnf(o.y);
    const float t1 = __fmaf_rn(w.z, __fmaf_rn(sx, w.x, o.x), 0.f);  // Wr (x) Or
    const float t2 = __fmaf_rn(w.w, __fmaf_rn(sy, w.y, o.y), 0.f);  // Wi (x) Oi
    const float t3 = __fmaf_rn(w.w, __fmaf_rn(sx, w.y, o.x), 0.f);  // Wi (x) Or
    const float t4 = __fmaf_rn(w.z, __fmaf_rn(sy, w.x, o.y), 0.f);  // Oi (x) Wr
    return make_float2(__fsub_rn(t1, t2), __fadd_rn(t3, t4));
}

// Stages b in [B0, W + 3) on the thread's 8 points r[j] (positions
// base | j << W); tlow = base mod 2^W.  tab holds the per-stage tables, stage
// b's 2^b entries starting at 2^b - 1.
template <int B0, int W>
__device__ __forceinline__ void nfft_stages(float2 (&r)[8], int tlow, const float4 *__restrict__ tab) {
#pragma unroll
    for (int b = B0; b < W + 3; ++b) {
        const int hb = b - W;
        const float4 *tb = tab + (1 << b) - 1;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j & (1 << hb)) continue;
            const int k = tlow | ((j & ((1 << hb) - 1)) << W);  // (base | j << W) mod 2^b
            const float4 w = tb[k];
            const float2 E = r[j];
            const float2 tt = cox_ready(w, r[j | (1 << hb)]);
            r[j] = make_float2(__fadd_rn(E.x, tt.x), __fadd_rn(E.y, tt.y));
            r[j | (1 << hb)] = make_float2(__fsub_rn(E.x, tt.x), __fsub_rn(E.y, tt.y));
        }
    }
}

template <int LOGN, int B0>
__device__ __forceinline__ void nfft_passes(float2 (&r)[8], float2 *s, int t, const float4 *__restrict__ tab,
                                            const float2 *__restrict__ xv, float2 *__restrict__ Xv, bool live) {
    if constexpr (B0 < LOGN) {
        constexpr int N = 1 << LOGN;
        constexpr int W = B0 + 3 <= LOGN ? B0 : LOGN - 3;  // window of 3 index bits
        constexpr bool first = B0 == 0, last = B0 + 3 >= LOGN;
        int base;
        if constexpr (first) {
            base = LOGN == 3 ? 0 : 8 * (int)(__brev((uint32_t)t) >> (32 - (LOGN - 3)));
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int m = ((j & 1) << 2) | (j & 2) | ((j >> 2) & 1);  // rev3(j)
                r[j] = live ? xv[t + m * (N / 8)] : make_float2(0.f, 0.f);
            }
        } else {
            base = (t & ((1 << W) - 1)) | ((t >> W) << (W + 3));
#pragma unroll
            for (int j = 0; j < 8; ++j) r[j] = s[swz(base | (j << W))];
        }
        nfft_stages<B0, W>(r, base & ((1 << W) - 1), tab);
        if constexpr (last) {
            // W = logN - 3 here, so base = t and positions are t + j N/8
            if (live)
#pragma unroll
                for (int j = 0; j < 8; ++j) Xv[base | (j << W)] = r[j];
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) s[swz(base | (j << W))] = r[j];
            __syncthreads();  // pass results visible before the next pass reads them
            nfft_passes<LOGN, B0 + 3>(r, s, t, tab, xv, Xv, live);
        }
    }
}

template <int LOGN>
struct NfftReg {
    static constexpr int N = 1 << LOGN;
    static constexpr int V = N >= 4096 ? 1 : 4096 / N;  // vectors per block
    static constexpr int threads = V * (N / 8);          // 512
    static constexpr size_t smem = (size_t)N * sizeof(float4) + (size_t)V * N * sizeof(float2);
};

template <int LOGN>
__global__ void __launch_bounds__(512) k_nfft_reg(const float2 *__restrict__ x, float2 *__restrict__ X,
                                                   const float2 *__restrict__ tw, int64_t batch) {
    using C = NfftReg<LOGN>;
    constexpr int N = C::N, V = C::V, tpv = N / 8;
    extern __shared__ __align__(16) float4 smem_nfft[];
    float4 *tab = smem_nfft;  // N - 1 entries used
    const int v = threadIdx.x / tpv, t = threadIdx.x - v * tpv;
    float2 *s = reinterpret_cast<float2 *>(smem_nfft + N) + v * N;
    // per-stage ready tables: entry 2^b - 1 + k holds W_N^(k 2^(logN-1-b))
    for (int e = threadIdx.x; e < N - 1; e += blockDim.x) {
        const int b = 31 - __clz(e + 1), k = e + 1 - (1 << b);
        const float2 w = __ldg(&tw[k << (LOGN - 1 - b)]);
        tab[e] = make_float4(fabsf(w.x), fabsf(w.y), sgnf(w.x), sgnf(w.y));
    }
    float2 r[8];
    for (int64_t g = blockIdx.x; g * V < batch; g += gridDim.x) {
        const int64_t vec = g * V + v;
        const bool live = vec < batch;
        __syncthreads();  // tables written; previous group's shared reads done
        nfft_passes<LOGN, 0>(r, s, t, tab, x + vec * N, X + vec * N, live);
    }
}

template <int LOGN>
cudaError_t launch_nfft_reg(const float2 *x, float2 *X, const float2 *tw, int64_t batch, int sm_count,
                            cudaStream_t s) {
    using C = NfftReg<LOGN>;
    static int occ = 0;  // resident blocks per SM, from the occupancy calculator
    if (occ == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_nfft_reg<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::smem);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nfft_reg<LOGN>, C::threads, C::smem);
        if (e != cudaSuccess) return e;
        occ = o > 0 ? o : 1;
    }
    const int64_t groups = (batch + C::V - 1) / C::V;
    const int64_t cap = (int64_t)sm_count * occ;
    const unsigned blocks = (unsigned)(groups < cap ? groups : cap);
    k_nfft_reg<LOGN><<<blocks, C::threads, C::smem, s>>>(x, X, tw, batch);
    return cudaGetLastError();
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
    if (N >= 8 && N <= 4096) {
        cudaError_t e;
        timer_begin(p, s);
        switch (logN) {
            case 3: e = launch_nfft_reg<3>(xi, Xo, p.tw32, batch, p.sm_count, s); break;
            case 4: e = launch_nfft_reg<4>(xi, Xo, p.tw32, batch, p.sm_count, s); break;
            case 5: e = launch_nfft_reg<5>(xi, Xo, p.tw32, batch, p.sm_count, s); break;
            case 6: e = launch_nfft_reg<6>(xi, Xo, p.tw32, batch, p.sm_count, s); break;
            case 7: e = launch_nfft_reg<7>(xi, Xo, p.tw32, batch, p.sm_count, s); break;
            case 8: e = launch_nfft_reg<8>(xi, Xo, p.tw32, batch, p.sm_count, s); break;
            case 9: e = launch_nfft_reg<9>(xi, Xo, p.tw32, batch, p.sm_count, s); break;
            case 10: e = launch_nfft_reg<10>(xi, Xo, p.tw32, batch, p.sm_count, s); break;
            case 11: e = launch_nfft_reg<11>(xi, Xo, p.tw32, batch, p.sm_count, s); break;
            default: e = launch_nfft_reg<12>(xi, Xo, p.tw32, batch, p.sm_count, s); break;
        }
        timer_end(p, s);
        *launches += 1;
        return e;
    }
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
