// fft_core.cuh -- radix-2 FFT machinery shared by the nonlinear FFT of Sec. 3
// (decimation in time and in frequency, Eq. 6 in every butterfly) and the
// ordinary FFT that Eq. 12b applies to the lag product.
//
// Butterflies ("ops"):
//   OpNL  t = W (x) O (Eq. 6), each real (x) rounded once -- the Sec. 3 recursion;
//   OpLin t = W O, the ordinary complex product -- the linear DFT of Eq. 12b.
// Decimation in time (DIT): bit-reversed input, stage b (butterfly distance
//   2^b, b = 0 .. L-1): t = op(W_2^(b+1)^k, O); E' = E + t; O' = E - t;
//   output in natural order.
// Decimation in frequency (DIF): natural input, stage b = L-1 .. 0:
//   E' = E + O; O' = op(W_2^(b+1)^k, E - O); output in bit-reversed order.
// k = (position of E) mod 2^b.  Every butterfly is evaluated in fp32 with one
// rounding per operation in exactly this order, so results are reproducible
// bit for bit; only data movement is optimised.
//
// Paths by size (L = log2 N): N <= 4 one thread per vector; 8 <= N <= 4096 one
// register kernel (all stages, one global read and write per point);
// 8192 <= N <= 65536 two kernels through an L2-sized workspace chunk: for DIT
// the register kernel runs stages 0 .. LA-1 on the 2^RB decimated
// sub-sequences and a register "tail" the last RB stages; for DIF a register
// "head" runs the first RB stages on natural-order data and the register kernel
// finishes each contiguous 2^LA block.
//
// The input is a "source" (a vector, or the Eq. 12a lag product generated on
// the fly) and the output a "sink" (all N bins in natural order, or the bins
// p0 .. p0 + nbins - 1 modulo N).
#pragma once

#include "internal.cuh"

#include <type_traits>

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

// The same lag product read from "comb-major" copies of s_surv and s_ref:
// element n of a length-N signal sits at (n mod C) N/C + n / C, C = 2^SB.  The
// first kernel of the two-kernel DIT path reads elements rev(c) + m C (one comb
// per sub-vector), which these copies make contiguous in m for both signals
// (n - l stays on one comb as m varies).  Same values as SrcLag.
struct SrcLagComb {
    const float2 *ssT, *srT;
    int N;
    int lag0;
    uint32_t flags;
    int sb;
    __device__ float2 operator()(int64_t v, int n) const {
        int64_t j = (int64_t)n - (lag0 + v);
        float2 ref = make_float2(0.f, 0.f);
        if (flags & NDFT_F_CIRCULAR_LAG) {
            j %= N;
            if (j < 0) j += N;
        }
        const int cmask = (1 << sb) - 1, ld = N >> sb;
        if (j >= 0 && j < N) {
            const int jj = (int)j;
            ref = srT[(jj & cmask) * ld + (jj >> sb)];
            if (!(flags & NDFT_F_NO_CONJ_REF)) ref.y = -ref.y;
        }
        return cox_f32(ssT[(n & cmask) * ld + (n >> sb)], ref);
    }
    SrcLagComb shift(int64_t a) const { return SrcLagComb{ssT, srT, N, (int)(lag0 + a), flags, sb}; }

    // One vector's elements n = rc + m 2^sb, m < N / 2^sb, as a row over m:
    // both combs and the reference offset are fixed per vector.  With
    // d = rc - (lag0 + v), the reference element n - (lag0 + v) = d + m 2^sb
    // lies on comb d mod 2^sb at index floor(d / 2^sb) + m, and is in range
    // iff 0 <= floor(d / 2^sb) + m < N / 2^sb (circular lags: d taken mod N
    // first and the index wrapped mod N / 2^sb).  Same values as operator().
    struct Row {
        const float2 *s, *r;  // s_surv's comb rc; the reference's comb for this lag
        int off, ld;          // reference index m + off; comb length
        bool circ, conj;
        __device__ float2 operator()(int m) const {
            float2 ref = make_float2(0.f, 0.f);
            const int k = m + off;
            if (circ || (unsigned)k < (unsigned)ld) {
                ref = r[k & (ld - 1)];
                if (conj) ref.y = -ref.y;
            }
            return cox_f32(s[m], ref);
        }
    };
    __device__ Row row(int64_t v, int rc) const {
        const int ld = N >> sb;
        const bool circ = (flags & NDFT_F_CIRCULAR_LAG) != 0;
        int64_t d = (int64_t)rc - ((int64_t)lag0 + v);
        if (circ) {
            d %= N;
            if (d < 0) d += N;
        }
        const int64_t q = d >> sb;  // floor(d / 2^sb)
        // beyond +-ld no m < ld reaches the reference (non-circular), so the
        // clamp keeps the index in int32 without changing any test
        const int off = (int)(q < -ld ? -ld : (q > ld ? ld : q));
        return Row{ssT + (int64_t)rc * ld, srT + (d & ((1 << sb) - 1)) * ld, off, ld, circ,
                   !(flags & NDFT_F_NO_CONJ_REF)};
    }
};

// Sources that offer a per-vector row over the first DIT kernel's comb.
template <class S>
struct HasCombRow : std::false_type {};
template <>
struct HasCombRow<SrcLagComb> : std::true_type {};

__global__ void k_comb_copy(const float2 *__restrict__ ss, const float2 *__restrict__ sr, float2 *__restrict__ ssT,
                            float2 *__restrict__ srT, int N, int sb) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int dst = (n & ((1 << sb) - 1)) * (N >> sb) + (n >> sb);
    ssT[dst] = ss[n];
    srT[dst] = sr[n];
}

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

// ---- butterflies -------------------------------------------------------------------
// sgn(v) as 1.0f, 0.0f or -1.0f.
__device__ __forceinline__ float sgnf(float v) {
    float g, l;
    asm("set.gt.f32.f32 %0, %1, 0f00000000;" : "=f"(g) : "f"(v));
    asm("set.lt.f32.f32 %0, %1, 0f00000000;" : "=f"(l) : "f"(v));
    return __fsub_rn(g, l);
}

// (sgn_mul, the two-instruction sgn of a data operand, is in internal.cuh:
// cox_ready only multiplies it by a twiddle magnitude and adds the operand
// back, and its outer fmas' +0 addends turn every zero into +0, so the result
// has the same bits as with sgnf.)

// Eq. 6 with the twiddle in "ready" form (|Re|, |Im|, sgn Re, sgn Im).  Each
// real a (x) b = sgn(a) sgn(b) (|a| + |b|) starts as the inner
// fma(sgn b, |a|, b) = sgn(b)(|a| + |b|), rounded once (round to nearest is
// symmetric); scaling it by sgn a (+-1 or 0) is exact, so the difference and
// the sum of Eq. 6 each take one more fma: Re = fma(sgn Wr, i1, -(Wi (x) Oi))
// with -(Wi (x) Oi) = fma(-sgn Wi, i2, +0), one rounding as in t1 - t2, and
// the +0 addend makes every zero come out +0, as the definition's 0 for a zero
// operand.  Same bits as cox_f32, signed zeros, subnormals, exact
// cancellations and the axis twiddles included.
__device__ __forceinline__ float2 cox_ready(float4 w, float2 o) {
    const float sx = sgn_mul(o.x), sy = sgn_mul(o.y);
    const float i1 = __fmaf_rn(sx, w.x, o.x);  // sgn Or (|Wr| + |Or|)
    const float i2 = __fmaf_rn(sy, w.y, o.y);  // sgn Oi (|Wi| + |Oi|)
    const float i3 = __fmaf_rn(sx, w.y, o.x);  // sgn Or (|Wi| + |Or|)
    const float i4 = __fmaf_rn(sy, w.x, o.y);  // sgn Oi (|Wr| + |Oi|)
    const float n2 = __fmaf_rn(-w.w, i2, 0.f);  // -(Wi (x) Oi)
    const float t4 = __fmaf_rn(w.z, i4, 0.f);   // Oi (x) Wr
    return make_float2(__fmaf_rn(w.z, i1, n2), __fmaf_rn(w.w, i3, t4));
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }

struct OpNL {
    __device__ static float4 prep(float2 w) { return make_float4(fabsf(w.x), fabsf(w.y), sgnf(w.x), sgnf(w.y)); }
    __device__ static float2 mul(float4 w, float2 o) { return cox_ready(w, o); }
};

// cox_ready for the two axis twiddles, same bits in 8 instructions instead of
// 12.  W = 1, ready form (1, 0, 1, 0): i1 = sgn Or + Or, i3 = 0 sgn Or + Or,
// n2 = -0 i2 + 0 = +0, t4 = i4 + 0 with i4 = sgn Oi + Oi, so
// Re = i1 + 0 and Im = 0 i3 + t4 = t4 (t4 is never -0):
//     W (x) O = (sgn Or + Or + 0, sgn Oi + Oi + 0).
// W = -j (table entry N/4: (+0, -1)), ready form (0, 1, 0, -1): n2 = i2 + 0
// with i2 = sgn Oi + Oi, t4 = 0 i4 + 0 = +0, Re = 0 i1 + n2 = n2,
// Im = -i3 + 0 with i3 = sgn Or + Or:
//     W (x) O = (sgn Oi + Oi + 0, -(sgn Or + Or) + 0).
// (fma(s, 1, o) is the rounded s + o; the + 0 turns a -0 into +0.)
__device__ __forceinline__ float2 cox_one(float2 o) {
    return make_float2(__fadd_rn(__fadd_rn(sgn_mul(o.x), o.x), 0.f), __fadd_rn(__fadd_rn(sgn_mul(o.y), o.y), 0.f));
}
__device__ __forceinline__ float2 cox_mj(float2 o) {
    return make_float2(__fadd_rn(__fadd_rn(sgn_mul(o.y), o.y), 0.f), __fadd_rn(-__fadd_rn(sgn_mul(o.x), o.x), 0.f));
}

struct OpLin {
    __device__ static float4 prep(float2 w) { return make_float4(w.x, w.y, 0.f, 0.f); }
    __device__ static float2 mul(float4 w, float2 o) {
        return make_float2(__fmaf_rn(w.x, o.x, -__fmul_rn(w.y, o.y)), __fmaf_rn(w.x, o.y, __fmul_rn(w.y, o.x)));
    }
};

template <class Op>
__device__ __forceinline__ void bfly_dit(float2 &e, float2 &o, float4 w) {
    const float2 E = e;
    const float2 tt = Op::mul(w, o);
    e = add2(E, tt);
    o = sub2(E, tt);
}

template <class Op>
__device__ __forceinline__ void bfly_dif(float2 &e, float2 &o, float4 w) {
    const float2 E = e, O = o;
    e = add2(E, O);
    o = Op::mul(w, sub2(E, O));
}

template <class Op, bool DIF>
__device__ __forceinline__ void bfly(float2 &e, float2 &o, float4 w) {
    if constexpr (DIF) bfly_dif<Op>(e, o, w);
    else bfly_dit<Op>(e, o, w);
}

// The nonlinear butterfly with the twiddle W = 1 (AXIS = 0) or W = -j (AXIS = 1).
template <bool DIF, int AXIS>
__device__ __forceinline__ void bfly_axis(float2 &e, float2 &o) {
    const float2 E = e;
    if constexpr (DIF) {
        const float2 O = o;
        e = add2(E, O);
        const float2 d = sub2(E, O);
        o = AXIS == 0 ? cox_one(d) : cox_mj(d);
    } else {
        const float2 tt = AXIS == 0 ? cox_one(o) : cox_mj(o);
        e = add2(E, tt);
        o = sub2(E, tt);
    }
}

// ---- N <= 4: one thread per vector ----------------------------------------------------
template <class Op, bool DIF, class Src, class Dst>
__global__ void k_fft_tiny(Src src, Dst dst, const float2 *__restrict__ tw, int logN, int64_t nvec) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvec) return;
    const int N = 1 << logN;
    float2 r[4];
    for (int p = 0; p < N; ++p) r[p] = src(v, DIF ? p : (int)bitrev(p, logN));
    for (int s = 0; s < logN; ++s) {
        const int b = DIF ? logN - 1 - s : s;
        for (int i0 = 0; i0 < N; ++i0) {
            if (i0 & (1 << b)) continue;
            const int k = i0 & ((1 << b) - 1);
            bfly<Op, DIF>(r[i0], r[i0 | (1 << b)], Op::prep(tw[k << (logN - 1 - b)]));
        }
    }
    for (int p = 0; p < N; ++p) dst(v, DIF ? (int)bitrev(p, logN) : p, r[p]);
}

// ---- 8 <= 2^LOGN <= 4096: register kernel ------------------------------------------
// Each thread keeps 8 points in registers and runs up to 3 radix-2 stages on
// them between shared-memory exchanges.  In a pass the thread's points are the
// positions base | j << W, j < 8: they differ in the 3 index bits [W, W + 3),
// so every stage whose butterfly distance 2^b lies in that window pairs two of
// the thread's own points.  DIT passes take windows upwards (W = 0, 3, ...,
// the last one clamped to LOGN - 3 and skipping stages already done), DIF
// passes downwards (the first one with W = LOGN - 3 taking only the top
// LOGN mod 3 stages when that is not 0, then W = ..., 3, 0), so that in both
// orders the stages b < 3 run in the W = 0 pass, where every twiddle index is
// a compile-time constant.
//
// Sub-vectors: with SB > 0 the kernel runs the 2^LOGN-point part of an NFFT of
// length 2^(LOGN+SB).  DIT: sub-vector q = o 2^SB + c is the transform of
// elements rev(c) + m 2^SB of source vector o (the first LOGN stages), written
// to dst(q, k).  DIF: sub-vector q reads src(q, m) (a contiguous block after
// the first SB stages) and its bin k is bin k 2^SB + rev(c) of vector o.
// SB = 0 is the whole transform.
//
// Data movement: the pass that touches global memory in bit-reversed order
// (the DIT load, the DIF store) remaps threads so that thread t takes the
// group at positions 8 rev(t) + j, i.e. natural indices t + rev3(j) 2^LOGN / 8,
// and the other end is natural order at positions t + j 2^LOGN / 8; both are
// coalesced.  Passes in between exchange through shared memory under an XOR
// swizzle of the low 4 index bits that keeps every exchange free of bank
// conflicts.  Twiddles sit in shared memory as one table per stage, indexed
// by k, prepared by the op, so a warp reads consecutive entries.
// swz is linear over GF(2) (shifts, masks and XORs of p's bits), and a
// thread's positions base | j << W have base and j << W on disjoint bits, so
// swz(base | j << W) = swz(base) ^ swz(j << W): one XOR with a constant per
// element once swz(base) is known.
__device__ __forceinline__ int swz(int p) { return p ^ ((p >> 4) & 15) ^ ((p >> 8) & 15) ^ ((p >> 3) & 8); }

__device__ __forceinline__ int rev3(int j) { return ((j & 1) << 2) | (j & 2) | ((j >> 2) & 1); }

template <int LOGN>
struct RegCfg {
    static constexpr int N = 1 << LOGN;
    static constexpr int V = N >= 4096 ? 1 : 4096 / N;  // sub-vectors per block
    static constexpr int threads = V * (N / 8);          // 512
    // exchange regions: two per sub-vector, used by alternate groups, where a
    // sub-vector's barrier is a named one over several warps and two blocks
    // per SM still fit (512 <= N <= 2048), else one (the loop-top barrier is
    // a __syncwarp for N <= 256, and measured cheaper than a second region)
    static constexpr int NB = N >= 512 && N <= 2048 ? 2 : 1;
    static constexpr size_t smem = (size_t)N * sizeof(float4) + (size_t)NB * V * N * sizeof(float2);
};

// Barrier over the N/8 threads of the calling thread's sub-vector.  Each
// sub-vector exchanges through a shared-memory region of its own, so the
// sub-vectors of a block need not wait for one another: __syncwarp when a
// sub-vector lies within one warp (N <= 256), else named barrier 1 + v over
// its warps (V <= 8 of them there; the ids are immediates so that the
// kernel reserves only the barriers it uses), the whole block when V = 1.
template <int ID, int TPV>
__device__ __forceinline__ void named_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(TPV) : "memory");
}
template <int LOGN>
__device__ __forceinline__ void vec_sync() {
    constexpr int tpv = (1 << LOGN) / 8, V = RegCfg<LOGN>::V;
    static_assert(V == 1 || tpv <= 32 || V <= 8, "one named barrier per sub-vector");
    if constexpr (V == 1) {
        __syncthreads();
    } else if constexpr (tpv <= 32) {
        __syncwarp();
    } else {
        switch (threadIdx.x / tpv) {  // uniform over each sub-vector's threads
            case 0: named_sync<1, tpv>(); break;
            case 1: named_sync<2, tpv>(); break;
            case 2: if constexpr (V > 2) named_sync<3, tpv>(); break;
            case 3: if constexpr (V > 3) named_sync<4, tpv>(); break;
            case 4: if constexpr (V > 4) named_sync<5, tpv>(); break;
            case 5: if constexpr (V > 5) named_sync<6, tpv>(); break;
            case 6: if constexpr (V > 6) named_sync<7, tpv>(); break;
            default: if constexpr (V > 7) named_sync<8, tpv>(); break;
        }
    }
}

// The barrier between two passes.  A position's writer and reader share
// their thread index above bit log2 G, with G = 2^W of the reader's window
// (DIT, after a pass other than the first) or of the writer's (DIF, before a
// pass other than the last): the exchange then closes over groups of G
// consecutive threads.  Where such a group is smaller than the sub-vector
// (G = 64 for 1024 <= N <= 4096: two warps) it may wait on named barrier
// 8 + g, above the sub-vector barriers 1 .. V (V <= 4 there); otherwise the
// sub-vector barrier.  Exchanges through the bit-reversed first (DIT) or
// last (DIF) pass span the sub-vector.  Measured on 2^26 points: N = 1024
// DIT 0.255 -> 0.250 ms (DIF unchanged), but N = 4096 0.297 -> 0.318 ms and
// the 4096-point passes of the 65536-point forms slower too, so only
// N = 1024 takes the group barriers.
template <int LOGN, int G>
__device__ __forceinline__ void pass_sync() {
    constexpr int tpv = (1 << LOGN) / 8, V = RegCfg<LOGN>::V;
    if constexpr (G >= tpv || LOGN != 10) {
        vec_sync<LOGN>();
    } else {
        static_assert(G == 64 && V <= 7 && RegCfg<LOGN>::threads / G <= 8, "group barriers 8 .. 15");
        switch (threadIdx.x / G) {  // uniform over each group's threads
            case 0: named_sync<8, G>(); break;
            case 1: named_sync<9, G>(); break;
            case 2: named_sync<10, G>(); break;
            case 3: named_sync<11, G>(); break;
            case 4: named_sync<12, G>(); break;
            case 5: named_sync<13, G>(); break;
            case 6: named_sync<14, G>(); break;
            default: named_sync<15, G>(); break;
        }
    }
}

// Stages b = B_HI - 1 .. B_LO (DIF, descending) or B_LO .. B_HI - 1 (DIT) on
// the thread's 8 points r[j] (positions base | j << W); tlow = base mod 2^W.
// tab holds the per-stage tables, stage b's 2^b entries starting at 2^b - 1.
template <class Op, bool DIF, int W, int B_LO, int B_HI>
__device__ __forceinline__ void reg_stages(float2 (&r)[8], int tlow, const float4 *__restrict__ tab) {
#pragma unroll
    for (int s = 0; s < B_HI - B_LO; ++s) {
        const int b = DIF ? B_HI - 1 - s : B_LO + s;
        const int hb = b - W;
        const float4 *tb = tab + (1 << b) - 1;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j & (1 << hb)) continue;
            const int k = tlow | ((j & ((1 << hb) - 1)) << W);  // (base | j << W) mod 2^b
            if constexpr (W == 0 && std::is_same<Op, OpNL>::value) {
                // tlow = 0 here, so k is known once the loops are unrolled: the
                // axis twiddles W^0 = 1 and W^(2^(b-1)) = -j take the short forms
                if (k == 0) {
                    bfly_axis<DIF, 0>(r[j], r[j | (1 << hb)]);
                    continue;
                }
                if (b > 0 && k == (1 << (b - 1))) {
                    bfly_axis<DIF, 1>(r[j], r[j | (1 << hb)]);
                    continue;
                }
            }
            bfly<Op, DIF>(r[j], r[j | (1 << hb)], tb[k]);
        }
    }
}

// DIT: pass starting at stage bit B0 (stages B0 .. min(B0 + 3, LOGN) - 1).
template <class Op, int LOGN, int SB, int B0, class Src, class Dst>
__device__ __forceinline__ void dit_passes(float2 (&r)[8], float2 *s, int t, const float4 *__restrict__ tab,
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
            if constexpr (SB > 0 && HasCombRow<Src>::value) {
                const auto row = src.row(o, rc);  // element rc + m 2^SB at m
#pragma unroll
                for (int j = 0; j < 8; ++j) r[j] = live ? row(t + rev3(j) * (N / 8)) : make_float2(0.f, 0.f);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    r[j] = live ? src(o, rc + ((t + rev3(j) * (N / 8)) << SB)) : make_float2(0.f, 0.f);
            }
        } else {
            base = (t & ((1 << W) - 1)) | ((t >> W) << (W + 3));
#pragma unroll
            for (int j = 0; j < 8; ++j) r[j] = s[swz(base) ^ swz(j << W)];
        }
        reg_stages<Op, false, W, B0, W + 3>(r, base & ((1 << W) - 1), tab);
        if constexpr (last) {
            // W = LOGN - 3 here, so base = t and positions are t + j N/8
            if (live)
#pragma unroll
                for (int j = 0; j < 8; ++j) dst(q, base | (j << W), r[j]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) s[swz(base) ^ swz(j << W)] = r[j];
            // pass results visible before the next pass (window WN) reads them
            constexpr int WN = B0 + 6 <= LOGN ? B0 + 3 : LOGN - 3;
            pass_sync<LOGN, first ? (1 << (LOGN - 3)) : (1 << WN)>();
            dit_passes<Op, LOGN, SB, B0 + 3>(r, s, t, tab, src, dst, q, live);
        }
    }
}

// DIF: pass ending below stage bit B1 (stages B1 - 1 .. LO).
template <class Op, int LOGN, int SB, int B1, class Src, class Dst>
__device__ __forceinline__ void dif_passes(float2 (&r)[8], float2 *s, int t, const float4 *__restrict__ tab,
                                           const Src &src, const Dst &dst, int64_t q, bool live) {
    if constexpr (B1 > 0) {
        constexpr int N = 1 << LOGN;
        constexpr bool first = B1 == LOGN;
        constexpr int W = B1 >= 3 ? B1 - 3 : 0;  // window of 3 index bits
        constexpr int LO = first && LOGN % 3 != 0 ? LOGN - LOGN % 3 : W;
        constexpr bool last = LO == 0;
        // positions base | j << W; the last pass remaps threads (see above)
        const int base = last ? 8 * (int)bitrev((uint32_t)t, LOGN - 3)
                              : (t & ((1 << W) - 1)) | ((t >> W) << (W + 3));
        if constexpr (first) {
#pragma unroll
            for (int j = 0; j < 8; ++j) r[j] = live ? src(q, base | (j << W)) : make_float2(0.f, 0.f);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) r[j] = s[swz(base) ^ swz(j << W)];
        }
        reg_stages<Op, true, W, LO, B1>(r, base & ((1 << W) - 1), tab);
        if constexpr (last) {
            // position 8 rev(t) + j holds bin rev(8 rev(t) + j) = rev3(j) N/8 + t
            if (live) {
                const int64_t o = q >> SB;
                const int rc = (int)bitrev((uint32_t)(q & ((1 << SB) - 1)), SB);
#pragma unroll
                for (int j = 0; j < 8; ++j) dst(o, ((t + rev3(j) * (N / 8)) << SB) + rc, r[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) s[swz(base) ^ swz(j << W)] = r[j];
            // pass results visible before the next pass reads them (that pass is
            // the last, bit-reversed one when its window starts at bit 0)
            constexpr bool next_last = LO <= 3;
            pass_sync<LOGN, next_last ? (1 << (LOGN - 3)) : (1 << W)>();
            dif_passes<Op, LOGN, SB, LO>(r, s, t, tab, src, dst, q, live);
        }
    }
}

template <class Op, bool DIF, int LOGN, int SB, class Src, class Dst>
__global__ void __launch_bounds__(512, 2) k_fft_reg(Src src, Dst dst, const float2 *__restrict__ tw, int64_t nsub) {
    using C = RegCfg<LOGN>;
    constexpr int N = C::N, V = C::V, tpv = N / 8;
    extern __shared__ __align__(16) float4 smem_fft[];
    float4 *tab = smem_fft;  // N - 1 entries used
    const int v = threadIdx.x / tpv, t = threadIdx.x - v * tpv;
    float2 *const s0 = reinterpret_cast<float2 *>(smem_fft + N) + v * N;
    // per-stage tables: entry 2^b - 1 + k holds W_2^(b+1)^k = tw[k 2^(LOGN+SB-1-b)]
    for (int e = threadIdx.x; e < N - 1; e += blockDim.x) {
        const int b = 31 - __clz(e + 1), k = e + 1 - (1 << b);
        tab[e] = Op::prep(__ldg(&tw[(k << (LOGN - 1 - b)) << SB]));
    }
    float2 r[8];
    __syncthreads();  // tables written
    int it = 0;
    for (int64_t g = blockIdx.x; g * V < nsub; g += gridDim.x, ++it) {
        const int64_t q = g * V + v;
        // With two regions, group it writes the one that group it - 2 read,
        // and every thread of the sub-vector has passed group it - 1's pass
        // barriers since (LOGN > 3: at least two passes); with one region the
        // sub-vector waits here for its reads of the previous group.
        float2 *s = s0;
        if constexpr (C::NB == 2) s += (it & 1) * V * N;
        else vec_sync<LOGN>();
        if constexpr (DIF) dif_passes<Op, LOGN, SB, LOGN>(r, s, t, tab, src, dst, q, q < nsub);
        else dit_passes<Op, LOGN, SB, 0>(r, s, t, tab, src, dst, q, q < nsub);
    }
}

template <class Op, bool DIF, int LOGN, int SB, class Src, class Dst>
cudaError_t launch_reg(Src src, Dst dst, const float2 *tw, int64_t nsub, int sm_count, cudaStream_t s) {
    using C = RegCfg<LOGN>;
    auto kern = k_fft_reg<Op, DIF, LOGN, SB, Src, Dst>;
    static int occ = 0;  // resident blocks per SM, from the occupancy calculator
    if (occ == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, C::threads, C::smem);
        if (e != cudaSuccess) return e;
        occ = o > 0 ? o : 1;
    }
    const int64_t groups = (nsub + C::V - 1) / C::V;
    const int64_t cap = (int64_t)sm_count * occ;
    const unsigned blocks = (unsigned)(groups < cap ? groups : cap);
    kern<<<blocks, C::threads, C::smem, s>>>(src, dst, tw, nsub);
    return cudaGetLastError();
}

// ---- 8192 <= N <= 65536: the RB stages at the far end -------------------------------
// Thread (vector o, u), u < 2^LA (LA = L - RB), holds positions u + j 2^LA,
// j < 2^RB, and runs stages LA .. L-1 (DIT tail: after the register kernel,
// reading the workspace, writing natural-order bins) or L-1 .. LA (DIF head:
// natural-order input, writing the workspace for the register kernel).  Loads
// and stores are coalesced over u.  Twiddles are read from the plan's table
// and prepared in registers.
template <class Op, bool DIF, int L, int RB, class Src, class Dst>
__global__ void __launch_bounds__(256) k_fft_edge(Src src, Dst dst, const float2 *__restrict__ tw, int64_t nvec) {
    constexpr int LA = L - RB, NA = 1 << LA, P = 1 << RB;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t o = gid >> LA;
    const int u = (int)(gid & (NA - 1));
    if (o >= nvec) return;
    float2 r[P];
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = src(o, u + (j << LA));
#pragma unroll
    for (int s = 0; s < RB; ++s) {
        const int hb = DIF ? RB - 1 - s : s;
        const int b = LA + hb;
        float4 w[P / 2];
#pragma unroll
        for (int qq = 0; qq < (1 << hb); ++qq) w[qq] = Op::prep(__ldg(&tw[(u | (qq << LA)) << (L - 1 - b)]));
#pragma unroll
        for (int j = 0; j < P; ++j) {
            if (j & (1 << hb)) continue;
            bfly<Op, DIF>(r[j], r[j | (1 << hb)], w[j & ((1 << hb) - 1)]);
        }
    }
#pragma unroll
    for (int j = 0; j < P; ++j) dst(o, u + (j << LA), r[j]);
}

// DIT tail when at most 2^LA bins are wanted (bins p0 .. p0 + nbins - 1 mod N):
// every position u then feeds exactly one wanted bin, u + m 2^LA, so a thread
// per wanted bin loads the 2^RB values of its u and runs only the butterflies
// that feed output m (2^RB - 1 of RB 2^(RB-1)): stages hb .. RB-1 mix index
// bits hb .. RB-1, so at stage hb those are the pairs whose bits below hb equal
// m's, and they all take the one twiddle of index m mod 2^hb.  The same
// butterflies on the same values as k_fft_edge, so the same bits.
template <class Op, int L, int RB>
__global__ void __launch_bounds__(256)
    k_fft_edge_bins(SrcVec src, DstBins dst, const float2 *__restrict__ tw, int64_t nvec) {
    constexpr int LA = L - RB, NA = 1 << LA, P = 1 << RB;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t o = gid / dst.nbins;
    const int t = (int)(gid - o * dst.nbins);
    if (o >= nvec) return;
    const int pbin = (dst.p0 + t) & dst.mask;  // the bin, mod N
    const int u = pbin & (NA - 1), m = pbin >> LA;
    float2 r[P];
#pragma unroll
    for (int j = 0; j < P; ++j) r[j] = src(o, u + (j << LA));
#pragma unroll
    for (int hb = 0; hb < RB; ++hb) {
        const int b = LA + hb;
        const int low = m & ((1 << hb) - 1);
        const float4 w = Op::prep(__ldg(&tw[(u | (low << LA)) << (L - 1 - b)]));
#pragma unroll
        for (int j = 0; j < P; ++j) {
            if (j & (1 << hb)) continue;
            if ((j & ((1 << hb) - 1)) != low) continue;  // does not feed output m
            bfly<Op, false>(r[j], r[j | (1 << hb)], w);
        }
    }
    float2 v = r[0];
#pragma unroll
    for (int j = 1; j < P; ++j)
        if (j == m) v = r[j];
    dst.A[o * dst.nbins + t] = v;
}

template <class Op, bool DIF, int L, int RB, class Src, class Dst>
cudaError_t run_two_pass(const Plan &p, Src src, Dst dst, int64_t nvec, cudaStream_t s, int *launches) {
    constexpr int LA = L - RB;
    float2 *Y = static_cast<float2 *>(p.nfft_ws);
    const int64_t ch = p.nfft_chunk;
    for (int64_t a0 = 0; a0 < nvec; a0 += ch) {
        const int64_t n = nvec - a0 < ch ? nvec - a0 : ch;
        const int64_t threads = n << LA;
        cudaError_t e;
        if constexpr (DIF) {
            k_fft_edge<Op, true, L, RB><<<(unsigned)(threads / 256), 256, 0, s>>>(
                src.shift(a0), DstVec{Y, (int64_t)1 << L}, p.tw32, n);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            e = launch_reg<Op, true, LA, RB>(SrcVec{Y, (int64_t)1 << LA}, dst.shift(a0), p.tw32, n << RB,
                                             p.sm_count, s);
            if (e != cudaSuccess) return e;
        } else {
            e = launch_reg<Op, false, LA, RB>(src.shift(a0), DstVec{Y, (int64_t)1 << LA}, p.tw32, n << RB,
                                              p.sm_count, s);
            if (e != cudaSuccess) return e;
            bool pruned = false;
            if constexpr (std::is_same_v<Dst, DstBins>) {
                if (dst.nbins <= (1 << LA)) {
                    const int64_t bt = n * dst.nbins;
                    k_fft_edge_bins<Op, L, RB><<<(unsigned)((bt + 255) / 256), 256, 0, s>>>(
                        SrcVec{Y, (int64_t)1 << L}, dst.shift(a0), p.tw32, n);
                    pruned = true;
                }
            }
            if (!pruned)
                k_fft_edge<Op, false, L, RB><<<(unsigned)(threads / 256), 256, 0, s>>>(
                    SrcVec{Y, (int64_t)1 << L}, dst.shift(a0), p.tw32, n);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        *launches += 2;
    }
    return cudaSuccess;
}

inline int log2i(int N) {
    int l = 0;
    while ((1 << l) < N) ++l;
    return l;
}

// Every path for N <= 65536 (fused source and sink); N > 4096 needs the
// plan's workspace chunk.
template <class Op, bool DIF, class Src, class Dst>
cudaError_t run_fft(const Plan &p, Src src, Dst dst, int64_t nvec, cudaStream_t s, int *launches) {
    const int L = log2i(p.d.n);
    if (nvec == 0) return cudaSuccess;
    if (L > 16 || (L > 12 && !p.nfft_ws)) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    timer_begin(p, s);
    if (L <= 2) {
        const int64_t blocks = (nvec + 255) / 256;
        if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
        k_fft_tiny<Op, DIF><<<(unsigned)blocks, 256, 0, s>>>(src, dst, p.tw32, L, nvec);
        e = cudaGetLastError();
        *launches += 1;
    } else if (L <= 12) {
        switch (L) {
            case 3: e = launch_reg<Op, DIF, 3, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 4: e = launch_reg<Op, DIF, 4, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 5: e = launch_reg<Op, DIF, 5, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 6: e = launch_reg<Op, DIF, 6, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 7: e = launch_reg<Op, DIF, 7, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 8: e = launch_reg<Op, DIF, 8, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 9: e = launch_reg<Op, DIF, 9, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 10: e = launch_reg<Op, DIF, 10, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            case 11: e = launch_reg<Op, DIF, 11, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
            default: e = launch_reg<Op, DIF, 12, 0>(src, dst, p.tw32, nvec, p.sm_count, s); break;
        }
        *launches += 1;
    } else {
        switch (L) {
            case 13: e = run_two_pass<Op, DIF, 13, 3>(p, src, dst, nvec, s, launches); break;
            case 14: e = run_two_pass<Op, DIF, 14, 3>(p, src, dst, nvec, s, launches); break;
            case 15: e = run_two_pass<Op, DIF, 15, 3>(p, src, dst, nvec, s, launches); break;
            default: e = run_two_pass<Op, DIF, 16, 4>(p, src, dst, nvec, s, launches); break;
        }
    }
    timer_end(p, s);
    return e;
}

// The three entry shapes every op/direction offers.
template <class Op, bool DIF>
cudaError_t fft_vectors(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s, int *launches) {
    const int N = p.d.n;
    return run_fft<Op, DIF>(p, SrcVec{static_cast<const float2 *>(x), N}, DstVec{static_cast<float2 *>(X), N},
                            batch, s, launches);
}

template <class Op, bool DIF>
cudaError_t fft_bins(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s, int *launches) {
    const int N = p.d.n;
    const DstBins dst{static_cast<float2 *>(X), N - 1, p.d.p0, p.d.nbins};
    return run_fft<Op, DIF>(p, SrcVec{static_cast<const float2 *>(x), N}, dst, batch, s, launches);
}

template <class Op, bool DIF>
cudaError_t fft_caf(const Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags, void *A,
                    cudaStream_t s, int *launches) {
    const int N = p.d.n;
    const float2 *ss = static_cast<const float2 *>(s_surv), *sr = static_cast<const float2 *>(s_ref);
    const DstBins dst{static_cast<float2 *>(A), N - 1, p.d.p0, p.d.nbins};
    const int L = log2i(N);
    if (!DIF && L > 12 && p.comb) {
        // two-kernel DIT: the first kernel reads one comb of stride 2^RB per sub-vector
        const int sb = L == 16 ? 4 : 3;
        float2 *ssT = p.comb, *srT = p.comb + N;
        k_comb_copy<<<(N + 255) / 256, 256, 0, s>>>(ss, sr, ssT, srT, N, sb);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        *launches += 1;
        return run_fft<Op, DIF>(p, SrcLagComb{ssT, srT, N, lag0, p.d.flags, sb}, dst, nlags, s, launches);
    }
    return run_fft<Op, DIF>(p, SrcLag{ss, sr, N, lag0, p.d.flags}, dst, nlags, s, launches);
}

}  // namespace
}  // namespace ndft
