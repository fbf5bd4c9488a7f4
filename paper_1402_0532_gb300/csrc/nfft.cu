// nfft.cu -- the nonlinear FFT of Sec. 3: radix-2 decimation in time with the
// twiddle product of every butterfly replaced by the operator of Eq. 6, and
// the cross-ambiguity surface of Eq. 12a evaluated through it.
//
// With the input in bit-reversed order, stage s (span L = 2^s) turns each pair
// of L/2-point NFFTs E, O into the L-point NFFT
//     t = W_L^k (x) O[k],   X[k] = E[k] + t,   X[k + L/2] = E[k] - t,
// W_L^k = W_N^(k N / L) read from the plan's fp32 table.  Every real (x) is
// rounded once and each add/subtract once, in this order, so the output is
// reproducible bit for bit.  Radix-4/8 regrouping would change the result
// (W1 (x) (W2 (x) v) != (W1 W2) (x) v), so only data movement is optimised.
//
// Sizes: N <= 4 one thread per vector; 8 <= N <= 4096 one register kernel
// (all stages, one global read and write per point); 8192 <= N <= 65536 two
// kernels -- the first runs stages 0 .. LA-1 on the 2^(logN-LA) decimated
// sub-sequences (each is an NFFT of its own, Sec. 3's recursion), the second
// the remaining 3 or 4 stages in registers -- through an L2-sized workspace
// chunk; larger N one launch per stage over global memory.
//
// The input of every path is a "source" (a vector, or the lag product of
// Eq. 12a generated on the fly) and its output a "sink" (all N bins in natural
// order, or the bins p0 .. p0 + nbins - 1 modulo N).
#include "internal.cuh"

namespace ndft {

namespace {

__device__ __forceinline__ uint32_t bitrev(uint32_t v, int bits) { return bits ? __brev(v) >> (32 - bits) : 0u; }

// ---- sources: element n (natural index) of vector v ------------------------------
struct SrcVec {
    const float2 *x;
    int64_t ld;
    __device__ float2 operator()(int64_t v, int n) const { return x[v * ld + n]; }
    SrcVec shift(int64_t a) const { return SrcVec{x + a * ld, ld}; }
};

// Lag product of Eq. 12a for lag lag0 + v: s_surv[n] (x) conj(s_ref[n - l]),
// s_ref zero outside [0, N) unless circular; the same fp32 expression as the
// direct and tensor-core forms.
struct SrcLag {
    const float2 *ss, *sr;
    int N;
    int lag0;
    uint32_t flags;
    __device__ float2 operator()(int64_t v, int n) const {
        int64_t j = (int64_t)n - (lag0 + v);
        float2 ref = make_float2(0.f, 0.f);
        if (flags & NDFT_F_CIRCULAR_LAG) {
            j %= N;
            if (j < 0) j += N;
        }
        if (j >= 0 && j < N) {
            ref = sr[j];
            if (!(flags & NDFT_F_NO_CONJ_REF)) ref.y = -ref.y;
        }
        return cox_f32(ss[n], ref);
    }
    SrcLag shift(int64_t a) const { return SrcLag{ss, sr, N, (int)(lag0 + a), flags}; }
};

// ---- sinks: output bin k (natural order) of vector v ----------------------------
struct DstVec {
    float2 *X;
    int64_t ld;
    __device__ void operator()(int64_t v, int k, float2 val) const { X[v * ld + k] = val; }
    DstVec shift(int64_t a) const { return DstVec{X + a * ld, ld}; }
};

// Bins p0 .. p0 + nbins - 1 taken modulo N (N a power of two: mask = N - 1).
struct DstBins {
    float2 *A;
    int mask;
    int p0;
    int nbins;
    __device__ void operator()(int64_t v, int k, float2 val) const {
        const int idx = (k - p0) & mask;
        if (idx < nbins) A[v * nbins + idx] = val;
    }
    DstBins shift(int64_t a) const { return DstBins{A + a * nbins, mask, p0, nbins}; }
};

// ---- the (x) butterfly ---------------------------------------------------------------
// sgn(v) as 1.0f, 0.0f or -1.0f.
__device__ __forceinline__ float sgnf(float v) {
    float g, l;
    asm("set.gt.f32.f32 %0, %1, 0f00000000;" : "=f"(g) : "f"(v));
    asm("set.lt.f32.f32 %0, %1, 0f00000000;" : "=f"(l) : "f"(v));
    return __fsub_rn(g, l);
}

// A twiddle in "ready" form: (|Re|, |Im|, sgn Re, sgn Im).
__device__ __forceinline__ float4 ready(float2 w) { return make_float4(fabsf(w.x), fabsf(w.y), sgnf(w.x), sgnf(w.y)); }

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

__device__ __forceinline__ void bfly(float2 &e, float2 &o, float4 w) {
    const float2 E = e;
    const float2 tt = cox_ready(w, o);
    e = make_float2(__fadd_rn(E.x, tt.x), __fadd_rn(E.y, tt.y));
    o = make_float2(__fsub_rn(E.x, tt.x), __fsub_rn(E.y, tt.y));
}

// ---- N <= 4: one thread per vector ----------------------------------------------------
template <class Src, class Dst>
__global__ void k_nfft_tiny(Src src, Dst dst, const float2 *__restrict__ tw, int logN, int64_t nvec) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvec) return;
    const int N = 1 << logN;
    float2 r[4];
    for (int p = 0; p < N; ++p) r[p] = src(v, (int)bitrev(p, logN));
    for (int b = 0; b < logN; ++b)
        for (int i0 = 0; i0 < N; ++i0) {
            if (i0 & (1 << b)) continue;
            const int k = i0 & ((1 << b) - 1);
            bfly(r[i0], r[i0 | (1 << b)], ready(tw[k << (logN - 1 - b)]));
        }
    for (int k = 0; k < N; ++k) dst(v, k, r[k]);
}

// ---- 8 <= 2^LOGN <= 4096: register kernel ------------------------------------------
// Each thread keeps 8 points in registers and runs up to 3 radix-2 stages on
// them between shared-memory exchanges.  In the pass that starts at stage bit
// B0 the thread's points differ in the 3 index bits [W, W + 3),
// W = min(B0, LOGN - 3), so every stage whose butterfly distance 2^b lies in
// that window pairs two of its own points; stages already done in earlier
// passes are skipped.  The butterflies and their order within each stage are
// those of the stage recursion, so results are identical bit for bit.
//
// The kernel transforms "sub-vectors": with SB > 0, sub-vector q = o 2^SB + c
// is the 2^LOGN-point NFFT of elements rev(c) + m 2^SB of source vector o --
// the first LOGN stages of an NFFT of length 2^(LOGN+SB) -- written to
// dst(q, k).  SB = 0 is the whole transform.
//
// Data movement: the first pass reads its points straight from the source
// (thread t of a sub-vector takes the group whose bit-reversed positions are
// 8 rev(t) + j, i.e. elements t + rev3(j) 2^LOGN / 8: coalesced for vectors),
// and the last pass writes straight to the sink (positions t + j 2^LOGN / 8,
// natural order).  Only the passes in between exchange through shared memory,
// under an XOR swizzle of the low 4 index bits that keeps every exchange free
// of bank conflicts.  Twiddles sit in shared memory as one table per stage,
// indexed by k, in ready form, so a warp reads consecutive entries.
__device__ __forceinline__ int swz(int p) { return p ^ ((p >> 4) & 15) ^ ((p >> 8) & 15) ^ ((p >> 3) & 8); }

// Stages b in [B0, W + 3) on the thread's 8 points r[j] (positions
// base | j << W); tlow = base mod 2^W.  tab holds the per-stage tables, stage
// b's 2^b entries starting at 2^b - 1.
template <int B0, int W>
__device__ __forceinline__ void reg_stages(float2 (&r)[8], int tlow, const float4 *__restrict__ tab) {
#pragma unroll
    for (int b = B0; b < W + 3; ++b) {
        const int hb = b - W;
        const float4 *tb = tab + (1 << b) - 1;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j & (1 << hb)) continue;
            const int k = tlow | ((j & ((1 << hb) - 1)) << W);  // (base | j << W) mod 2^b
            bfly(r[j], r[j | (1 << hb)], tb[k]);
        }
    }
}

template <int LOGN, int SB, int B0, class Src, class Dst>
__device__ __forceinline__ void reg_passes(float2 (&r)[8], float2 *s, int t, const float4 *__restrict__ tab,
                                           const Src &src, const Dst &dst, int64_t q, bool live) {
    if constexpr (B0 < LOGN) {
        constexpr int N = 1 << LOGN;
        constexpr int W = B0 + 3 <= LOGN ? B0 : LOGN - 3;  // window of 3 index bits
        constexpr bool first = B0 == 0, last = B0 + 3 >= LOGN;
        int base;
        if constexpr (first) {
            base = 8 * (int)bitrev((uint32_t)t, LOGN - 3);
            const int64_t o = q >> SB;
            const int rc = (int)bitrev((uint32_t)(q & ((1 << SB) - 1)), SB);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int m = ((j & 1) << 2) | (j & 2) | ((j >> 2) & 1);  // rev3(j)
                r[j] = live ? src(o, rc + ((t + m * (N / 8)) << SB)) : make_float2(0.f, 0.f);
            }
        } else {
            base = (t & ((1 << W) - 1)) | ((t >> W) << (W + 3));
#pragma unroll
            for (int j = 0; j < 8; ++j) r[j] = s[swz(base | (j << W))];
        }
        reg_stages<B0, W>(r, base & ((1 << W) - 1), tab);
        if constexpr (last) {
            // W = LOGN - 3 here, so base = t and positions are t + j N/8
            if (live)
#pragma unroll
                for (int j = 0; j < 8; ++j) dst(q, base | (j << W), r[j]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) s[swz(base | (j << W))] = r[j];
            __syncthreads();  // pass results visible before the next pass reads them
            reg_passes<LOGN, SB, B0 + 3>(r, s, t, tab, src, dst, q, live);
        }
    }
}

template <int LOGN>
struct RegCfg {
    static constexpr int N = 1 << LOGN;
    static constexpr int V = N >= 4096 ? 1 : 4096 / N;  // sub-vectors per block
    static constexpr int threads = V * (N / 8);          // 512
    static constexpr size_t smem = (size_t)N * sizeof(float4) + (size_t)V * N * sizeof(float2);
};

template <int LOGN, int SB, class Src, class Dst>
__global__ void __launch_bounds__(512, 2) k_nfft_reg(Src src, Dst dst, const float2 *__restrict__ tw, int64_t nsub) {
    using C = RegCfg<LOGN>;
    constexpr int N = C::N, V = C::V, tpv = N / 8;
    extern __shared__ __align__(16) float4 smem_nfft[];
    float4 *tab = smem_nfft;  // N - 1 entries used
    const int v = threadIdx.x / tpv, t = threadIdx.x - v * tpv;
    float2 *s = reinterpret_cast<float2 *>(smem_nfft + N) + v * N;
    // per-stage ready tables: entry 2^b - 1 + k holds W_2^(b+1)^k = tw[k 2^(LOGN+SB-1-b)]
    for (int e = threadIdx.x; e < N - 1; e += blockDim.x) {
        const int b = 31 - __clz(e + 1), k = e + 1 - (1 << b);
        tab[e] = ready(__ldg(&tw[(k << (LOGN - 1 - b)) << SB]));
    }
    float2 r[8];
    for (int64_t g = blockIdx.x; g * V < nsub; g += gridDim.x) {
        const int64_t q = g * V + v;
        __syncthreads();  // tables written; previous group's shared reads done
        reg_passes<LOGN, SB, 0>(r, s, t, tab, src, dst, q, q < nsub);
    }
}

template <int LOGN, int SB, class Src, class Dst>
cudaError_t launch_reg(Src src, Dst dst, const float2 *tw, int64_t nsub, int sm_count, cudaStream_t s) {
    using C = RegCfg<LOGN>;
    static int occ = 0;  // resident blocks per SM, from the occupancy calculator
    if (occ == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_nfft_reg<LOGN, SB, Src, Dst>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nfft_reg<LOGN, SB, Src, Dst>, C::threads, C::smem);
        if (e != cudaSuccess) return e;
        occ = o > 0 ? o : 1;
    }
    const int64_t groups = (nsub + C::V - 1) / C::V;
    const int64_t cap = (int64_t)sm_count * occ;
    const unsigned blocks = (unsigned)(groups < cap ? groups : cap);
    k_nfft_reg<LOGN, SB, Src, Dst><<<blocks, C::threads, C::smem, s>>>(src, dst, tw, nsub);
    return cudaGetLastError();
}

// ---- 8192 <= N <= 65536: the last RB stages ------------------------------------------
// Y holds, per vector, the 2^RB NFFTs of length 2^LA (LA = L - RB) of the
// first kernel, sub-vector c at offset c 2^LA -- exactly the bit-reversed-order
// array after stage LA - 1.  Thread (vector o, u) holds positions u + j 2^LA,
// j < 2^RB, runs stages LA .. L-1 on them in registers and writes the natural-
// order bins u + j 2^LA.  Loads and stores are coalesced over u.
template <int L, int RB, class Dst>
__global__ void __launch_bounds__(256) k_nfft_tail(const float2 *__restrict__ Y, Dst dst,
                                                    const float2 *__restrict__ tw, int64_t nvec) {
    constexpr int LA = L - RB, NA = 1 << LA, P = 1 << RB;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t o = gid >> LA;
    const int u = (int)(gid & (NA - 1));
    if (o >= nvec) return;
    const float2 *y = Y + (o << L);
    float2 r[P];
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = y[u + (j << LA)];
#pragma unroll
    for (int hb = 0; hb < RB; ++hb) {
        const int b = LA + hb;
        float4 w[P / 2];
#pragma unroll
        for (int qq = 0; qq < (1 << hb); ++qq) w[qq] = ready(__ldg(&tw[(u | (qq << LA)) << (L - 1 - b)]));
#pragma unroll
        for (int j = 0; j < P; ++j) {
            if (j & (1 << hb)) continue;
            bfly(r[j], r[j | (1 << hb)], w[j & ((1 << hb) - 1)]);
        }
    }
#pragma unroll
    for (int j = 0; j < P; ++j) dst(o, u + (j << LA), r[j]);
}

template <int L, int RB, class Src, class Dst>
cudaError_t run_two_pass(const Plan &p, Src src, Dst dst, int64_t nvec, cudaStream_t s, int *launches) {
    constexpr int LA = L - RB;
    float2 *Y = static_cast<float2 *>(p.nfft_ws);
    const int64_t ch = p.nfft_chunk;
    for (int64_t a0 = 0; a0 < nvec; a0 += ch) {
        const int64_t n = nvec - a0 < ch ? nvec - a0 : ch;
        cudaError_t e = launch_reg<LA, RB>(src.shift(a0), DstVec{Y, (int64_t)1 << LA}, p.tw32, n << RB,
                                           p.sm_count, s);
        if (e != cudaSuccess) return e;
        const int64_t threads = n << LA;
        k_nfft_tail<L, RB><<<(unsigned)(threads / 256), 256, 0, s>>>(Y, dst.shift(a0), p.tw32, n);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 2;
    }
    return cudaSuccess;
}

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

int log2i(int N) {
    int l = 0;
    while ((1 << l) < N) ++l;
    return l;
}

// Every path for N <= 65536 (fused source and sink).
template <class Src, class Dst>
cudaError_t run_nfft(const Plan &p, Src src, Dst dst, int64_t nvec, cudaStream_t s, int *launches) {
    const int L = log2i(p.d.n);
    if (nvec == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    timer_begin(p, s);
    if (L <= 2) {
        const int64_t blocks = (nvec + 255) / 256;
        if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
        k_nfft_tiny<<<(unsigned)blocks, 256, 0, s>>>(src, dst, p.tw32, L, nvec);
        e = cudaGetLastError();
        *launches += 1;
    } else if (L <= 12) {
        switch (L) {
            case 3: e = launch_reg<3, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 4: e = launch_reg<4, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 5: e = launch_reg<5, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 6: e = launch_reg<6, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 7: e = launch_reg<7, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 8: e = launch_reg<8, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 9: e = launch_reg<9, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 10: e = launch_reg<10, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 11: e = launch_reg<11, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            default: e = launch_reg<12, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
        }
        *launches += 1;
    } else {
        switch (L) {
            case 13: e = run_two_pass<13, 3>(p, src, dst, nvec, s, launches); break;
            case 14: e = run_two_pass<14, 3>(p, src, dst, nvec, s, launches); break;
            case 15: e = run_two_pass<15, 3>(p, src, dst, nvec, s, launches); break;
            default: e = run_two_pass<16, 4>(p, src, dst, nvec, s, launches); break;
        }
    }
    timer_end(p, s);
    return e;
}

}  // namespace

size_t nfft_ws_bytes(const ndft_desc &d, int64_t *chunk) {
    *chunk = 0;
    const int64_t N = d.n;
    if (d.prec != NDFT_PREC_FP32 || N < 8192 || N > 65536 || (N & (N - 1))) return 0;
    int64_t want = d.max_batch;
    if (d.form == NDFT_FORM_NFFT && d.max_lags > want) want = d.max_lags;
    if (want <= 0) return 0;
    int64_t ch = (int64_t)(kNfftChunkBytes / (N * (int64_t)sizeof(float2)));
    if (ch < 1) ch = 1;
    if (ch > want) ch = want;
    *chunk = ch;
    return (size_t)ch * N * sizeof(float2);
}

cudaError_t launch_nfft(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s, int *launches) {
    const int N = p.d.n;
    const int logN = log2i(N);
    if (batch == 0) return cudaSuccess;
    const float2 *xi = static_cast<const float2 *>(x);
    float2 *Xo = static_cast<float2 *>(X);
    if (N <= 4096 || (N <= 65536 && p.nfft_ws))
        return run_nfft(p, SrcVec{xi, N}, DstVec{Xo, N}, batch, s, launches);
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
    const int N = p.d.n;
    if (N > 4096 && !p.nfft_ws) return cudaErrorInvalidValue;
    const DstBins dst{static_cast<float2 *>(X), N - 1, p.d.p0, p.d.nbins};
    return run_nfft(p, SrcVec{static_cast<const float2 *>(x), N}, dst, batch, s, launches);
}

cudaError_t launch_nfft_caf(const Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags, void *A,
                            cudaStream_t s, int *launches) {
    const int N = p.d.n;
    if (N > 4096 && !p.nfft_ws) return cudaErrorInvalidValue;
    const SrcLag src{static_cast<const float2 *>(s_surv), static_cast<const float2 *>(s_ref), N, lag0, p.d.flags};
    const DstBins dst{static_cast<float2 *>(A), N - 1, p.d.p0, p.d.nbins};
    return run_nfft(p, src, dst, nlags, s, launches);
}

}  // namespace ndft
