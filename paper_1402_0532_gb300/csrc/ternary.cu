// ternary.cu -- the tensor-core form of the NDFT / nonlinear CAF.
//
// Real a (x) b = sgn(a b)(|a| + |b|) equals sgn(b) a + sgn(a) b exactly (both
// addends are exact), so through Eq. 6 a complex (x) is sigma(a) b + a sigma(b)
// with sigma(v) = sgn(v_r) + j sgn(v_i).  The NDFT of Eq. 8 (and the CAF of
// Eq. 12a, the NDFT of each lag product) becomes two dense contractions:
//     X = S v + F sigma(v),   F[p][i] = W^(p i),   S = sigma(F)  (ternary).
// As one real GEMM, row 2p (Re X[p]) and row 2p+1 (Im X[p]) of the operand A
// hold, per sample i, eight K entries that pair with the eight B entries
//     B = [v_hi_r, v_lo_r, v_hi_i, v_lo_i, s_r, s_r, s_i, s_i]      (s = sigma(v))
//     A(re) = [S_r, S_r, -S_i, -S_i, F_hi_r, F_lo_r, -F_hi_i, -F_lo_i]
//     A(im) = [S_i, S_i,  S_r,  S_r, F_hi_i, F_lo_i,  F_hi_r,  F_lo_r]
// with v = v_hi + v_lo and F = F_hi + F_lo split into bf16 pairs; the ternary
// entries are exact in bf16 and the products accumulate in fp32 (TMEM).
//
// Kernel layout (one persistent CTA per SM, 448 threads):
//   warp 0      TMA producer: B tiles (256 columns x 64 K) from the packed
//               buffer, 128-byte swizzle, one mbarrier per stage;
//   warp 1      TMEM allocator and single-thread tcgen05.mma issuer;
//   warps 2-9   A producers: generate the 256 x 64 A tile of each stage in
//               shared memory: F by complex rotation of each twiddle, re-seeded
//               from a 2-level cos/sin table every 16 K blocks; the sign
//               pattern S by range tests on the integer twiddle index, so its
//               zeros are exact; then fence.proxy.async and arrive;
//   warps 10-13 epilogue: tcgen05.ld the two 128 x 256 fp32 accumulators and
//               fold them into the output or split-K partials by bulk tensor
//               stores / adds, releasing row half 0 as soon as it is read.
// The 2-SM pair variant (k_ternary_gemm_pair) and the adjoint modes are
// described where they are defined.
// Every mbarrier wait is bounded; a timeout records NDFT_E_TIMEOUT in the
// plan's error word and the CTA drains and exits.
#include "internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace ndft {

namespace {

constexpr int TN = 256;            // columns per tile
constexpr int KB = 64;             // bf16 K per stage = 8 samples x 8 entries
constexpr int B_BYTES = TN * 128;  // 32 KiB
constexpr int R_LO = 256;          // angle split r = r_hi * 256 + r_lo
constexpr int kMaxN = 1 << 18;
constexpr int kMaxThi = kMaxN / R_LO + 2;
constexpr int kGenWarps = 8;
// the conjugate-paired contraction generates twice the twiddles per MMA of the
// unpaired one and runs twice the A-producer warps (4 per SM sub-partition) to
// hide their latency
constexpr int kGenWarpsPair = 16;
// A tiles loaded from a plan-time table (ATAB) need no producer warps
__host__ __device__ constexpr int gemm_gen_warps(bool pair, bool atab = false) {
    return atab ? 0 : (pair ? kGenWarpsPair : kGenWarps);
}
__host__ __device__ constexpr int gemm_threads(bool pair, bool atab = false) {
    return (2 + gemm_gen_warps(pair, atab) + 4) * 32;
}
constexpr int kMaxSplit = 32;
constexpr int kChunk = 64;  // K blocks per TMEM accumulation chain (512 samples)
// paired form: 64 K blocks of 16 samples (1024 samples, the same 256 MMA K
// steps per chain as the unpaired default).  The tensor core's truncating fp32
// accumulation makes the error grow with the K steps of a chain: measured on
// the N = 2^18 NDFT of CN(0,1) vectors (the worst case found), chains of 32 /
// 64 / 128 / 256 paired blocks give 2.5e-6 / 4.0e-6 / 8.2e-6 / 1.6e-5 of max|X|
// (the unpaired form 2.6e-6 / 4.9e-6 / 8.4e-6 / 1.7e-5 at the same K steps)
constexpr int kChunkPair = 64;
// largest plan-time A table of the paired contraction (512 MiB for a
// 65536-sample surface of 1024 bins)
constexpr size_t kAtabMaxBytes = (size_t)2 << 30;
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz


// One problem: the single transform of a plan, or one CPI of a batched plan.
struct Problem {
    int32_t N, p0, nbins, ncols;
    int32_t kblocks, nsplit, mtiles, ntiles;
    int64_t b_row0;        // first 128-byte row of this problem's packed B
    int64_t out_off;       // floats from the launch's output base to this problem's output / partials
    int64_t ld;            // floats per column of out (= 2 * nbins)
    int64_t split_stride;  // floats between split partials
    const float2 *ang;     // two-level table: [nth] (r_hi) then [256] (r_lo)
    int32_t nth;
    int32_t a_ld;          // paired A table: rows per K block (the padded row count)
    int32_t crow0;         // batched: first column of this problem in the output tensor map
    // adjoint mode: s_ref and the lag window of the forward call
    const float2 *sref;
    int32_t lag0;
    uint32_t flags;
};

struct Unit {
    int32_t prob, mt, nt, split;
};

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the barrier did not complete within kWaitCycles or
// another role already gave up (abort flag).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int32_t *abort_flag,
                                          int32_t *err) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            dev_set_error(err, kDevTimeout);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_b(uint32_t dst, const CUtensorMap *map, int32_t row, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
    // K-major, 128-byte swizzle: start >> 4, LBO (unused) = 1, SBO = 1024 B, version 1, layout 2
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// kind::f16, D fp32, A/B bf16, both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 2-CTA cluster helpers (the pair tile): this CTA's rank and a cluster-wide barrier.
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ void red_add_f32(float *addr, float v) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void gen_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kGenWarps * 32) : "memory"); }
template <int GW>
__device__ __forceinline__ void gen_bar_n() { asm volatile("bar.sync 1, %0;" ::"n"(GW * 32) : "memory"); }

// Bulk tensor copies of a staged [32 columns][128 rows] fp32 block to the
// output map at {row, column, split}: plain store, or element-wise add in L2.
__device__ __forceinline__ void tma_store_out(const CUtensorMap *map, uint32_t src, int m, int col, int split) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(m), "r"(col), "r"(split), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void tma_reduce_out(const CUtensorMap *map, uint32_t src, int m, int col, int split) {
    asm volatile("cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(m), "r"(col), "r"(split), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ---- unit decoding -------------------------------------------------------------
struct Work {
    Problem P;
    int mt, nt, kb0, kb1;
    int split;
    int64_t out_off;  // floats from the launch's output base
};

// Unit u of the launch: from the work list of a batched plan, or (single
// problem) split-major with m-tiles fastest.
__device__ __forceinline__ Work decode(int64_t u, const Problem &single, const Problem *probs, const Unit *units) {
    Work w;
    if (units) {
        const Unit un = units[u];
        w.P = probs[un.prob];
        w.mt = un.mt;
        w.nt = un.nt;
        w.kb0 = (int)((int64_t)un.split * w.P.kblocks / w.P.nsplit);
        w.kb1 = (int)((int64_t)(un.split + 1) * w.P.kblocks / w.P.nsplit);
        w.split = un.split;
        w.out_off = w.P.out_off + (int64_t)un.split * w.P.split_stride;
    } else {
        w.P = single;
        const int64_t tiles = (int64_t)single.mtiles * single.ntiles;
        const int split = (int)(u / tiles);
        const int64_t t = u - (int64_t)split * tiles;
        w.mt = (int)(t % single.mtiles);
        w.nt = (int)(t / single.mtiles);
        w.kb0 = (int)((int64_t)split * single.kblocks / single.nsplit);
        w.kb1 = (int)((int64_t)(split + 1) * single.kblocks / single.nsplit);
        w.split = split;
        w.out_off = single.out_off + (int64_t)split * single.split_stride;
    }
    return w;
}

// ---- A generation: one (bin, sample) pair -> rows 2 pl and 2 pl + 1 ------------
// u = 4 m, m = (p i) mod N; theta = 2 pi m / N = q pi/2 + a with q = floor(u / N),
// a = (pi/2) r / N, r = u - q N.  cos a, sin a from the two-level table (explicit
// shared loads: the aligned dynamic shared-memory base is reached through
// integer arithmetic, so plain pointer loads would take the generic path).
// The producers compute all of their pairs of a K block before storing any.
__device__ __forceinline__ float2 lds_f2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

// The twiddle W = cos(theta) - j sin(theta) at u = 4 ((p i) mod N) from the
// two-level table (full plane; exact 0 / +-1 on the axes).  Used to seed the
// rotation below and for the rotation step itself.
__device__ __forceinline__ float2 tw_table(uint32_t u, uint32_t N, uint32_t thi, uint32_t tlo) {
    const uint32_t q = (u >= N) + (u >= 2 * N) + (u >= 3 * N);
    const uint32_t r = u - q * N;
    const float2 h = lds_f2(thi + (r >> 8) * 8u);
    const float2 l = lds_f2(tlo + (r & (R_LO - 1)) * 8u);
    const float c = fmaf(h.x, l.x, -(h.y * l.y));
    const float s = fmaf(h.y, l.x, h.x * l.y);
    //   q0: ( c, -s)   q1: (-s, -c)   q2: (-c,  s)   q3: ( s,  c)
    return q == 0u ? make_float2(c, -s) : q == 1u ? make_float2(-s, -c) : q == 2u ? make_float2(-c, s)
                                                                            : make_float2(s, c);
}

// The same from the table in global memory (cached in L1).
__device__ __forceinline__ float2 tw_table_g(uint32_t u, uint32_t N, const float2 *__restrict__ ang, int nth) {
    const uint32_t q = (u >= N) + (u >= 2 * N) + (u >= 3 * N);
    const uint32_t r = u - q * N;
    const float2 h = __ldg(ang + (r >> 8));
    const float2 l = __ldg(ang + nth + (r & (R_LO - 1)));
    const float c = fmaf(h.x, l.x, -(h.y * l.y));
    const float s = fmaf(h.y, l.x, h.x * l.y);
    return q == 0u ? make_float2(c, -s) : q == 1u ? make_float2(-s, -c) : q == 2u ? make_float2(-c, s)
                                                                            : make_float2(s, c);
}

// sigma(W) at u = 4 ((p i) mod N) in [0, 4N) as bf16 pairs, exact: Re W = cos
// is < 0 for N < u < 3N and 0 at u = N, 3N; Im W = -sin is < 0 for 0 < u < 2N
// and 0 at u = 0, 2N (the integer quadrant rule written as range tests).
__device__ __forceinline__ void sign_bits(uint32_t u, uint32_t N, uint32_t &sr2, uint32_t &si2) {
    constexpr uint32_t P1 = 0x3F803F80u, NEG = 0x80008000u;
    const bool neg_r = (u - (N + 1u)) < (2u * N - 1u);  // unsigned: false for u <= N
    const bool nz_r = (u != N) && (u != 3u * N);
    const bool neg_i = u < 2u * N;
    const bool nz_i = (u != 0u) && (u != 2u * N);
    sr2 = nz_r ? (P1 | (neg_r ? NEG : 0u)) : 0u;
    si2 = nz_i ? (P1 | (neg_i ? NEG : 0u)) : 0u;
}

// The 8 K entries of one (bin, sample) pair: the Re row's to re[], the Im
// row's to im[] (layout in the file header), with F taken from a given value
// of W (the rotated twiddle) and the ternary signs S from the integer quadrant
// rule on u, so the signs stay exact (0 on the axes) whatever the rounding of W.
__device__ __forceinline__ void gen_pair_w(uint32_t u, uint32_t N, float2 W, uint4 &re, uint4 &im) {
    uint32_t sr, si;  // [S_r, S_r], [S_i, S_i]
    sign_bits(u, N, sr, si);
    const __nv_bfloat162 hi2 = __floats2bfloat162_rn(W.x, W.y);
    const __nv_bfloat162 lo2 = __floats2bfloat162_rn(W.x - __low2float(hi2), W.y - __high2float(hi2));
    const uint32_t uh = *reinterpret_cast<const uint32_t *>(&hi2);
    const uint32_t ul = *reinterpret_cast<const uint32_t *>(&lo2);
    const uint32_t wr = __byte_perm(uh, ul, 0x5410);  // [F_hi_r, F_lo_r]
    const uint32_t wi = __byte_perm(uh, ul, 0x7632);  // [F_hi_i, F_lo_i]
    re = make_uint4(sr, si ^ 0x80008000u, wr, wi ^ 0x80008000u);
    im = make_uint4(si, sr, wi, wr);
}

// Conjugate-paired form, one 16-byte chunk of a row = samples a and a + 1 of
// the K block, in the K order [S(a), S(a+1), S(a), S(a+1), F_hi(a), F_hi(a+1),
// F_lo(a), F_lo(a+1)] (the packed B chunk pairs [v_hi, v_lo, sigma, sigma] in
// the same order), so every word is one bf16x2 conversion of two samples.
// The twiddle index is carried as an exact integer-valued float uf = 4 ((c i)
// mod N) < 2^20, and the exact signs come from it by range arithmetic:
//     sgn Re W = sgn((uf - N)(uf - 3N)),   sgn Im W = sgn(uf (uf - 2N)),
// both factors exact integers, so the product is 0 exactly on the axes and
// otherwise at least 1 in magnitude: clamping it to [-1, 1] gives the sign.
__device__ __forceinline__ float sgn_clamp(float x) { return fminf(fmaxf(x, -1.f), 1.f); }

__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// hi and lo words of the bf16 split of two values
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
    hi = bf2(x0, x1);
    lo = bf2(x0 - __uint_as_float(hi << 16), x1 - __uint_as_float(hi & 0xFFFF0000u));
}

struct PackProb {
    int64_t a_off;    // elements from the launch's first input base: x (NDFT) or s_surv (CAF)
    int64_t r_off;    // elements from the launch's second input base: s_ref (CAF)
    int32_t N, lag0, ncols, kblocks;
    int64_t ldx;      // row stride of x
    int64_t row0;     // first packed row
};

// sgn(v) in two instructions: 1.0f where v != 0 (set.ne) with v's sign bit
// copied in, so +-1, or a zero of v's sign for a zero v.  As a factor it is
// exact; a zero of either sign contributes nothing to a nonzero sum.
__device__ __forceinline__ float sgn_or_zero(float v) {
    float nz;
    asm("set.ne.f32.f32 %0, %1, 0f00000000;" : "=f"(nz) : "f"(v));
    return __uint_as_float(__float_as_uint(nz) | (__float_as_uint(v) & 0x80000000u));
}

// Eq. 6 for the lag product s (x) c, c = conj(r) (or r with NDFT_F_NO_CONJ_REF):
// Re = s_r (x) c_r - s_i (x) c_i, Im = s_i (x) c_r + s_r (x) c_i.  Each real
// a (x) b = sgn(a) sgn(b) (|a| + |b|) is the inner fma(sgn b, |a|, b), rounded
// once, times sgn a (exact); the difference and the sum then take one fma
// each, Re = fma(sgn s_r, i1, n2) with n2 = -(s_i (x) c_i) exact (its +0
// addend turns a zero into +0), one rounding as in t1 - t2.  Same values as
// the four products and the subtraction written out; zeros come out +0 or of
// either sign where the definition gives 0.
__device__ __forceinline__ float2 lag_ox(float2 s, float2 r, bool conj) {
    const float cr = r.x, ci = conj ? -r.y : r.y;
    const float gsr = sgn_or_zero(s.x), gsi = sgn_or_zero(s.y), gcr = sgn_or_zero(cr), gci = sgn_or_zero(ci);
    const float i1 = __fmaf_rn(gcr, fabsf(s.x), cr);  // sgn c_r (|s_r| + |c_r|)
    const float i2 = __fmaf_rn(gci, fabsf(s.y), ci);  // sgn c_i (|s_i| + |c_i|)
    const float i3 = __fmaf_rn(gcr, fabsf(s.y), cr);  // sgn c_r (|s_i| + |c_r|)
    const float i4 = __fmaf_rn(gsr, fabsf(ci), s.x);  // sgn s_r (|c_i| + |s_r|)
    const float n2 = __fmaf_rn(-gsi, i2, 0.f);        // -(s_i (x) c_i)
    const float t4 = __fmaf_rn(gci, i4, 0.f);         // c_i (x) s_r
    return make_float2(__fmaf_rn(gsr, i1, n2), __fmaf_rn(gsi, i3, t4));
}

// ---- the conjugate-paired B operand, two samples of one input column ----------
// Samples i (even) and i + 1 of column `lag` - lag0: the CAF lag products
// v = s_surv[i] (x) conj(s_ref[i - lag]) (Eq. 12a; zero where i - lag falls
// outside the reference, wrapped with circular lags) or, for the NDFT, the
// input row itself (`a` = that row); zero past N.  `vec`: `a` is 16-byte
// aligned, so the two samples are one 16-byte load.
// The loads: v0, v1 = the inputs at i, i + 1 and (CAF) r0, r1 = the reference
// at i - lag, i + 1 - lag; pair_combine forms the lag products from them.
__device__ __forceinline__ void pair_loads(const float2 *__restrict__ a, const float2 *__restrict__ r, int i, int N,
                                           int64_t lag, bool caf, bool circ, bool vec, float2 &v0, float2 &v1,
                                           float2 &r0, float2 &r1) {
    const float2 zero = make_float2(0.f, 0.f);
    v0 = v1 = r0 = r1 = zero;
    if (i + 1 < N && vec) {
        const float4 s2 = *reinterpret_cast<const float4 *>(a + i);
        v0 = make_float2(s2.x, s2.y);
        v1 = make_float2(s2.z, s2.w);
    } else {
        if (i < N) v0 = a[i];
        if (i + 1 < N) v1 = a[i + 1];
    }
    if (caf) {
        int64_t j = (int64_t)i - lag;
        if (circ) {
            j %= N;
            if (j < 0) j += N;
        }
        int64_t j1 = j + 1;
        if (circ && j1 == N) j1 = 0;
        if (i < N && j >= 0 && j < N) r0 = r[j];
        if (i + 1 < N && j1 >= 0 && j1 < N) r1 = r[j1];
    }
}
__device__ __forceinline__ void pair_combine(bool caf, bool conj, float2 r0, float2 r1, float2 &v0, float2 &v1) {
    if (caf) {
        v0 = lag_ox(v0, r0, conj);
        v1 = lag_ox(v1, r1, conj);
    }
}
__device__ __forceinline__ void pair_samples(const float2 *__restrict__ a, const float2 *__restrict__ r, int i, int N,
                                             int64_t lag, bool caf, bool conj, bool circ, bool vec, float2 &v0,
                                             float2 &v1) {
    float2 r0, r1;
    pair_loads(a, r, i, N, lag, caf, circ, vec, v0, v1, r0, r1);
    pair_combine(caf, conj, r0, r1, v0, v1);
}

// The (col, r) and (col, i) chunks of v0, v1 ([v_hi, v_lo, sigma, sigma] as
// bf16x2 words of the two samples) and their terms v + sigma(v) of the
// column's bin-0 sum.
__device__ __forceinline__ void pair_chunks(float2 v0, float2 v1, uint4 &re, uint4 &im, float &dr, float &di) {
    uint32_t hr, lr, hi, li;
    split2(v0.x, v1.x, hr, lr);
    split2(v0.y, v1.y, hi, li);
    const float g0r = sgn_or_zero(v0.x), g1r = sgn_or_zero(v1.x), g0i = sgn_or_zero(v0.y),
                g1i = sgn_or_zero(v1.y);
    const uint32_t sr2 = bf2(g0r, g1r), si2 = bf2(g0i, g1i);
    re = make_uint4(hr, lr, sr2, sr2);
    im = make_uint4(hi, li, si2, si2);
    dr = (v0.x + g0r) + (v1.x + g1r);
    di = (v0.y + g0i) + (v1.y + g1i);
}

// The B operand of the 2-SM pair tile: loaded by TMA from the packed buffer
// (kBTma, packed by k_pack_pair before the launch), formed in shared memory
// (kBForm), or packed into the buffer by the tile's own producer warps ahead
// of its TMA loads (kBAhead).
constexpr int kBTma = 0, kBForm = 1, kBAhead = 2;

// What the producer warps read and write for kBForm / kBAhead.
struct BGen {
    PackProb pp;
    const float2 *a;  // launch's first input base (x or s_surv)
    const float2 *r;  // s_ref (CAF)
    float2 *dc;       // bin-0 sums: kBForm [nsplit][ncols], kBAhead [nsplit * jmax][ncols]
    uint32_t flags;
    int32_t caf;
    // kBAhead: work items (split s, block j of 16 K blocks from the split's
    // first, 64-column block cx), jmax blocks per split, ncx column blocks
    uint4 *B;         // the packed buffer
    int32_t *ctr;     // [1 + (s jmax + j) ncx + cx]: item state, 0 free, 1 claimed, 2 packed
    int64_t nitems;
    int32_t jmax, ncx;
    int32_t look;     // items the packers may run ahead of their CTA's TMA loads
};

// The R and I chunks of one frequency for samples a and a + 1 (twiddles Wa, Wb
// at indices ua, ub).
__device__ __forceinline__ void gen_conj_chunk(float ua, float ub, float2 Wa, float2 Wb, float fN, uint4 &re,
                                               uint4 &im) {
    const float sra = sgn_clamp((ua - fN) * (ua - 3.f * fN)), srb = sgn_clamp((ub - fN) * (ub - 3.f * fN));
    const float sia = sgn_clamp(ua * (ua - 2.f * fN)), sib = sgn_clamp(ub * (ub - 2.f * fN));
    const uint32_t SR = bf2(sra, srb), SI = bf2(sia, sib);
    uint32_t hr, lr, hi, li;
    split2(Wa.x, Wb.x, hr, lr);
    split2(Wa.y, Wb.y, hi, li);
    re = make_uint4(SR, SR, hr, lr);
    im = make_uint4(SI, SI, hi, li);
}

// W <- W * R (fp32 complex product)
__device__ __forceinline__ float2 cmul_f2(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -(a.y * b.y)), fmaf(a.x, b.y, a.y * b.x));
}

// A producers advance each (bin, sample) twiddle by W^(8p) per K block and
// re-seed it from the table every kReseed blocks: the table gathers (bank
// conflicted, the largest share of the shared-memory wavefronts) drop to
// 1/kReseed, and the rotation's drift stays near 1e-6, below the 2^-17
// resolution of the bf16 hi + lo split of F.
constexpr int kReseed = 16;

// ---- adjoint A generation: sample i, bins p and p + 1 -> rows 2 i and 2 i + 1 --// ---- adjoint A generation: sample i, bins p and p + 1 -> rows 2 i and 2 i + 1 --
// The adjoint contraction G_l[i] = sum_p conj(S[p][i]) dA[l][p] runs with rows =
// (sample, Re/Im), columns = lags, K = bins x [dA_hi_r, dA_lo_r, dA_hi_i,
// dA_lo_i].  Per bin the Re row holds [S_r, S_r, S_i, S_i] and the Im row
// [-S_i, -S_i, S_r, S_r] (conj(S) dA = S_r a_r + S_i a_i + j (S_r a_i - S_i a_r)),
// S = sigma(W^(p i)) read off u = 4 ((p i) mod N) by the integer quadrant rule
// (exact zeros on the axes), as bf16 pairs.
__device__ __forceinline__ void adj_signs(uint32_t u, uint32_t N, uint32_t &sr2, uint32_t &si2) {
    sign_bits(u, N, sr2, si2);
}

// Rows 2 pl (Re) and 2 pl + 1 (Im), 16-byte chunk t of the 128-byte row, in the
// 128-byte-swizzled K-major layout the MMA descriptors expect.
// One row's 16-byte chunk t, in the same swizzled layout.
__device__ __forceinline__ void store_row(uint32_t a_stage, int row, int t, const uint4 &v) {
    sts128(a_stage + (uint32_t)row * 128u + (((uint32_t)t ^ ((uint32_t)row & 7u)) << 4), v.x, v.y, v.z, v.w);
}

__device__ __forceinline__ void store_pair(uint32_t a_stage, int pl, int t, const uint4 &re, const uint4 &im) {
    const uint32_t row_re = 2u * pl, row_im = row_re + 1u;
    const uint32_t base_re = a_stage + row_re * 128u + (((uint32_t)t ^ (row_re & 7u)) << 4);
    const uint32_t base_im = a_stage + row_im * 128u + (((uint32_t)t ^ (row_im & 7u)) << 4);
    sts128(base_re, re.x, re.y, re.z, re.w);
    sts128(base_im, im.x, im.y, im.z, im.w);
}

// MH row halves of 128 rows per tile.  MH = 2: 256 x 256 tile, one TMEM
// accumulator pair (all 512 columns), the MMA waits while a finished chain is
// folded out.  MH = 1: 128 x 256 tile, two 256-column accumulators used in
// turn, so the fold of one chain overlaps the MMAs of the next.
template <int MH>
struct Tile {
    static constexpr int kRows = 128 * MH;
    static constexpr int kABytes = kRows * 128;
    static constexpr int kStages = MH == 1 ? 4 : 3;
    static constexpr int kBufs = MH == 1 ? 2 : 1;
    static constexpr size_t kSmemA = 0;
    static constexpr size_t kSmemB = kSmemA + (size_t)kStages * kABytes;
    static constexpr size_t kSmemTab = kSmemB + (size_t)kStages * B_BYTES;
    static constexpr size_t kSmemStage = (kSmemTab + (size_t)(kMaxThi + R_LO) * sizeof(float2) + 127) / 128 * 128;
    static constexpr size_t kSmemBar = kSmemStage + 4 * 4096;  // per epilogue warp 2 x [16 cols][32 rows] fp32
    static constexpr size_t kSmemTotal = kSmemBar + 160 + 1024;  // barriers, flags, alignment slack
};

// The conjugate-paired contraction: the 256-row tile without the twiddle table
// in shared memory (its producers read the table through L1, a re-seed every
// 16 K blocks) and with 4 KB fold-out buffers, two per epilogue warp, so that
// each bulk copy moves 32 columns.
struct TileP {
    static constexpr int kRows = 256;
    static constexpr int kABytes = kRows * 128;
    static constexpr int kStages = 3;
    static constexpr int kBufs = 1;
    static constexpr size_t kSmemA = 0;
    static constexpr size_t kSmemB = kSmemA + (size_t)kStages * kABytes;
    static constexpr size_t kSmemStage = kSmemB + (size_t)kStages * B_BYTES;
    static constexpr size_t kSmemTab = kSmemStage;  // unused
    static constexpr size_t kSmemBar = kSmemStage + 4 * 8192;  // per epilogue warp 2 x [32 cols][32 rows] fp32
    static constexpr size_t kSmemTotal = kSmemBar + 160 + 1024;
};
static_assert(TileP::kSmemTotal <= 232448, "shared memory of one CTA");

template <bool PAIR, int MH>
struct TileOf {
    using type = Tile<MH>;
};
template <int MH>
struct TileOf<true, MH> {
    using type = TileP;
};

// ADJ selects the adjoint contractions (rows = samples, columns = lags, K =
// bins): 1 folds G into dL/ds_surv in the epilogue, 2 stores G itself (the
// forward epilogue on a [lags][2N] fp32 output).
// ATAB (paired rows only): the A tiles come by TMA from a table the plan built
// (rows [K block][padded rows] of 128 bytes) instead of producer warps: the
// forward's R/I rows, or the paired adjoint's sign rows.
template <int MH, bool BT, int ADJ, bool PAIR = false, bool ATAB = false>
__global__ void __launch_bounds__(gemm_threads(PAIR, ATAB), 1)
    k_ternary_gemm(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap omap, int out_tma,
                   Problem single, const Problem *__restrict__ probs, const Unit *__restrict__ units, int64_t nunits,
                   int chunk, int starve, float *__restrict__ out_base, int32_t *err,
                   const __grid_constant__ CUtensorMap amap) {
    static_assert(ADJ == 0 || (MH == 2 && !BT), "the adjoint runs on the 256-row tile");
    static_assert(!PAIR || (MH == 2 && !BT), "the conjugate-paired form runs on the 256-row tile");
    static_assert(!ATAB || PAIR, "the A tables are for the paired contractions");
    constexpr int GW = gemm_gen_warps(PAIR, ATAB);  // A-producer warps: warps 2 .. 2 + GW - 1
    constexpr int EPI0 = 2 + GW;              // epilogue warps EPI0 .. EPI0 + 3 -> TMEM lane quarters warp % 4
    using T = typename TileOf<PAIR, MH>::type;
    constexpr int STG = T::kStages;
    constexpr int NB = T::kBufs;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    float2 *s_thi = reinterpret_cast<float2 *>(smem + T::kSmemTab);
    float2 *s_tlo = s_thi + kMaxThi;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + T::kSmemBar);
    uint64_t *empty = full + STG;
    uint64_t *tmem_full = empty + STG;    // [NB]
    uint64_t *tmem_empty = tmem_full + NB;  // [NB]
    // MH = 2: the epilogue also signals when it has read row half 0 (TMEM
    // columns 0 .. 255), so the next chain's half-0 MMAs can start while it
    // still reads half 1
    uint64_t *tmem_half0 = tmem_empty + NB;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(tmem_half0 + 1);
    volatile int32_t *s_abort = reinterpret_cast<volatile int32_t *>(s_tmem + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t a_base = smem_u32(smem + T::kSmemA), b_base = smem_u32(smem + T::kSmemB);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STG; ++s) {
            mbar_init(&full[s], 1 + GW);
            mbar_init(&empty[s], 1);  // one MMA commit
        }
        for (int b = 0; b < NB; ++b) {
            mbar_init(&tmem_full[b], 1);
            mbar_init(&tmem_empty[b], 4);
        }
        mbar_init(tmem_half0, 4);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
        if constexpr (ATAB) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&amap)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                const Work w = decode(u, single, probs, units);
                for (int kb = w.kb0; kb < w.kb1; ++kb) {
                    if (!(ok = mbar_wait(&empty[stage], phase ^ 1u, s_abort, err))) break;
                    if (starve) continue;  // tests: the stage never fills, every wait runs out
                    mbar_arrive_tx(&full[stage], B_BYTES + (ATAB ? (uint32_t)T::kABytes : 0u));
                    const int64_t row = w.P.b_row0 + (int64_t)kb * w.P.ncols + (int64_t)w.nt * TN;
                    tma_load_b(b_base + stage * B_BYTES, &tmap, (int32_t)row, &full[stage]);
                    if constexpr (ATAB) {
                        const int64_t arow = (int64_t)kb * w.P.a_ld + (int64_t)w.mt * T::kRows;
                        tma_load_b(a_base + stage * T::kABytes, &amap, (int32_t)arow, &full[stage]);
                    }
                    if (++stage == STG) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, chain = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                const Work w = decode(u, single, probs, units);
                // one accumulation chain per chunk of `chunk` K blocks; the epilogue
                // folds each chain into the destination in fp32 (round to nearest)
                for (int c0 = w.kb0; c0 < w.kb1 && ok; c0 += chunk, ++chain) {
                    const int c1 = min(c0 + chunk, w.kb1);
                    const uint32_t buf = chain % NB, tpar = (chain / NB) & 1u;
                    const uint32_t d0 = tmem + buf * (uint32_t)TN;
                    int kb = c0;
                    if constexpr (MH == 2) {
                        // Half 0 of the accumulator is free first: run its MMAs for the
                        // stages already loaded while the epilogue still reads half 1 of
                        // the previous chain, then half 1's for the same stages.  Each
                        // half still accumulates its K blocks in order.
                        if (!(ok = mbar_wait(tmem_half0, tpar ^ 1u, s_abort, err))) break;
                        tc_fence_after();
                        const int npro = min(STG, c1 - c0);
                        int st = stage;
                        uint32_t ph = phase;
                        for (int q = 0; q < npro; ++q) {
                            if (!(ok = mbar_wait(&full[st], ph, s_abort, err))) break;
                            tc_fence_after();
                            const uint32_t a_st = a_base + st * T::kABytes, b_st = b_base + st * B_BYTES;
#pragma unroll
                            for (int k = 0; k < KB / 16; ++k)
                                umma(d0, umma_desc(a_st + k * 32), umma_desc(b_st + k * 32), (q > 0 || k > 0) ? 1u : 0u);
                            if (++st == STG) {
                                st = 0;
                                ph ^= 1u;
                            }
                        }
                        if (!ok) break;
                        if (!(ok = mbar_wait(&tmem_empty[buf], tpar ^ 1u, s_abort, err))) break;
                        tc_fence_after();
                        for (int q = 0; q < npro; ++q) {
                            const uint32_t a_st = a_base + stage * T::kABytes, b_st = b_base + stage * B_BYTES;
#pragma unroll
                            for (int k = 0; k < KB / 16; ++k)
                                umma(d0 + TN, umma_desc(a_st + 128 * 128 + k * 32), umma_desc(b_st + k * 32),
                                     (q > 0 || k > 0) ? 1u : 0u);
                            umma_commit(&empty[stage]);
                            if (++stage == STG) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                        kb = c0 + npro;
                    } else {
                        if (!(ok = mbar_wait(&tmem_empty[buf], tpar ^ 1u, s_abort, err))) break;
                        tc_fence_after();
                    }
                    for (; kb < c1; ++kb) {
                        if (!(ok = mbar_wait(&full[stage], phase, s_abort, err))) break;
                        tc_fence_after();
                        const uint32_t a_st = a_base + stage * T::kABytes, b_st = b_base + stage * B_BYTES;
#pragma unroll
                        for (int k = 0; k < KB / 16; ++k) {
                            const uint64_t bd = umma_desc(b_st + k * 32);
                            const uint32_t acc = (kb > c0 || k > 0) ? 1u : 0u;
#pragma unroll
                            for (int h = 0; h < MH; ++h)
                                umma(d0 + h * TN, umma_desc(a_st + h * 128 * 128 + k * 32), bd, acc);
                        }
                        umma_commit(&empty[stage]);
                        if (++stage == STG) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    umma_commit(&tmem_full[buf]);
                }
            }
        }
        __syncwarp();
    } else if (warp < EPI0) {
        // ---------------- A producers ----------------
        constexpr int PPT = 2 * MH;      // (bin, sample) pairs per thread per K block
        const int g = threadIdx.x - 64;  // 0 .. 32 GW - 1
        const int t = g & 7, pg = g >> 3;
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        if constexpr (ATAB) {
            // no producer warps: the TMA warp loads the A tiles from the table
        } else if constexpr (ADJ != 0 && PAIR) {
            // Conjugate-paired adjoint: one row per sample i, K = frequencies
            // c = p0, p0 + 1, ... (4 entries each, [S_r, S_r, S_i, S_i] of
            // S = sigma(W^(c i)), against the packed [u_hi, u_lo, v_hi, v_lo]
            // of the two columns of each lag); thread (pg, t) makes rows
            // pg + 4 GW j, frequencies 2 t and 2 t + 1 of each K block (16
            // frequencies), signs by the integer quadrant rule.
            constexpr int RPT = 256 / (4 * GW);
            for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                const Work w = decode(u, single, probs, units);
                const uint32_t N = (uint32_t)w.P.N;
                uint32_t ua[RPT], ub[RPT], dd[RPT];
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const int64_t i = ((int64_t)w.mt * 256 + pg + 4 * GW * j) % (int64_t)N;  // sample
                    int64_t c0 = ((int64_t)w.P.p0 + (int64_t)w.kb0 * 16 + 2 * t) % (int64_t)N;
                    if (c0 < 0) c0 += N;
                    const int64_t c1 = c0 + 1 == N ? 0 : c0 + 1;
                    ua[j] = 4u * (uint32_t)((c0 * i) % N);
                    ub[j] = 4u * (uint32_t)((c1 * i) % N);
                    dd[j] = 4u * (uint32_t)((16 * i) % N);
                }
                for (int kb = w.kb0; kb < w.kb1; ++kb) {
                    if (!(ok = mbar_wait(&empty[stage], phase ^ 1u, s_abort, err))) break;
                    const uint32_t a_st = a_base + stage * T::kABytes;
#pragma unroll
                    for (int j = 0; j < RPT; ++j) {
                        uint32_t sra, sia, srb, sib;
                        sign_bits(ua[j], N, sra, sia);
                        sign_bits(ub[j], N, srb, sib);
                        store_row(a_st, pg + 4 * GW * j, t, make_uint4(sra, sia, srb, sib));
                        ua[j] += dd[j];
                        if (ua[j] >= 4u * N) ua[j] -= 4u * N;
                        ub[j] += dd[j];
                        if (ub[j] >= 4u * N) ub[j] -= 4u * N;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full[stage]);
                    if (++stage == STG) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        } else if constexpr (ADJ != 0) {
            for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                const Work w = decode(u, single, probs, units);
                const uint32_t N = (uint32_t)w.P.N;
                uint32_t ua[PPT], ub[PPT], dd[PPT];
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const int64_t i = (int64_t)w.mt * (T::kRows / 2) + pg + 32 * j;  // sample
                    int64_t pa = ((int64_t)w.P.p0 + (int64_t)w.kb0 * 16 + 2 * t) % (int64_t)N;
                    if (pa < 0) pa += N;
                    const int64_t pb = pa + 1 == N ? 0 : pa + 1;
                    ua[j] = 4u * (uint32_t)((pa * (i % N)) % N);
                    ub[j] = 4u * (uint32_t)((pb * (i % N)) % N);
                    dd[j] = 4u * (uint32_t)((16 * (i % N)) % N);
                }
                for (int kb = w.kb0; kb < w.kb1; ++kb) {
                    if (!(ok = mbar_wait(&empty[stage], phase ^ 1u, s_abort, err))) break;
                    const uint32_t a_st = a_base + stage * T::kABytes;
#pragma unroll
                    for (int j = 0; j < PPT; ++j) {
                        uint32_t sra, sia, srb, sib;
                        adj_signs(ua[j], N, sra, sia);
                        adj_signs(ub[j], N, srb, sib);
                        const uint4 re = make_uint4(sra, sia, srb, sib);
                        const uint4 im = make_uint4(sia ^ 0x80008000u, sra, sib ^ 0x80008000u, srb);
                        store_pair(a_st, pg + 32 * j, t, re, im);
                        ua[j] += dd[j];
                        if (ua[j] >= 4u * N) ua[j] -= 4u * N;
                        ub[j] += dd[j];
                        if (ub[j] >= 4u * N) ub[j] -= 4u * N;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full[stage]);
                    if (++stage == STG) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        } else if constexpr (PAIR) {
            // Conjugate-paired rows: slot k of the unit is the frequency
            // c = p0 + k (p0 = the first paired frequency); its R row (2 k) and
            // I row (2 k + 1) hold the signs and bf16 hi + lo parts of Re and
            // Im F, F = W^(c i), in the chunk order of gen_conj_chunk.  A K
            // block is 16 samples; thread (pg, t) makes slots pg + 4 GW j,
            // samples 2 t and 2 t + 1 of it, each twiddle advanced by
            // W^(16 c) per K block and re-seeded from the table every kReseed
            // blocks; the index advances in exact float arithmetic.
            constexpr int SPT = 32 / GW;  // slots per thread: pg + 4 GW j
            for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
                const Work w = decode(u, single, probs, units);
                if (!ok) break;
                const uint32_t N = (uint32_t)w.P.N;
                const float fN = (float)N, f4N = 4.f * fN;
                const float2 *ang = w.P.ang;
                const int nth = w.P.nth;
                float ua[SPT], ub[SPT], dd[SPT];  // exact integers < 2^20
                float2 wa[SPT], wb[SPT], rot[SPT];
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    const int k = w.mt * 128 + pg + 4 * GW * j;  // slot
                    int64_t c = ((int64_t)w.P.p0 + k) % (int64_t)N;
                    if (c < 0) c += N;
                    const int64_t i0 = (int64_t)w.kb0 * 16 + 2 * t;
                    const uint32_t d4 = 4u * (uint32_t)((16 * c) % (int64_t)N);
                    ua[j] = (float)(4u * (uint32_t)((c * (i0 % (int64_t)N)) % (int64_t)N));
                    ub[j] = (float)(4u * (uint32_t)((c * ((i0 + 1) % (int64_t)N)) % (int64_t)N));
                    dd[j] = (float)d4;
                    rot[j] = tw_table_g(d4, N, ang, nth);  // W^(16 c)
                }
                for (int kb = w.kb0; kb < w.kb1; ++kb) {
                    if (!(ok = mbar_wait(&empty[stage], phase ^ 1u, s_abort, err))) break;
                    const uint32_t a_st = a_base + stage * T::kABytes;
                    const bool seed = ((kb - w.kb0) % kReseed) == 0;
                    uint4 vre[SPT], vim[SPT];
#pragma unroll
                    for (int j = 0; j < SPT; ++j) {
                        if (seed) {
                            wa[j] = tw_table_g((uint32_t)ua[j], N, ang, nth);
                            wb[j] = tw_table_g((uint32_t)ub[j], N, ang, nth);
                        }
                        gen_conj_chunk(ua[j], ub[j], wa[j], wb[j], fN, vre[j], vim[j]);
                        wa[j] = cmul_f2(wa[j], rot[j]);
                        wb[j] = cmul_f2(wb[j], rot[j]);
                        ua[j] += dd[j];
                        if (ua[j] >= f4N) ua[j] -= f4N;
                        ub[j] += dd[j];
                        if (ub[j] >= f4N) ub[j] -= f4N;
                    }
#pragma unroll
                    for (int j = 0; j < SPT; ++j) store_pair(a_st, pg + 4 * GW * j, t, vre[j], vim[j]);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full[stage]);
                    if (++stage == STG) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        } else
        for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
            const Work w = decode(u, single, probs, units);
            gen_bar();  // every producer is done with the previous table
            for (int e = g; e < w.P.nth + R_LO; e += kGenWarps * 32) {
                const float2 v = w.P.ang[e];
                if (e < w.P.nth) s_thi[e] = v;
                else s_tlo[e - w.P.nth] = v;
            }
            gen_bar();
            if (!ok) continue;
            const uint32_t N = (uint32_t)w.P.N;
            const uint32_t thi = smem_u32(s_thi), tlo = smem_u32(s_tlo);
            uint32_t uu[PPT], dd[PPT];
            float2 wv[PPT], rot[PPT];
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int k = w.mt * (T::kRows / 2) + pg + 32 * j;  // bin index
                int64_t pm = ((int64_t)w.P.p0 + k) % (int64_t)N;
                if (pm < 0) pm += N;
                const int64_t i0 = (int64_t)w.kb0 * 8 + t;
                uu[j] = 4u * (uint32_t)((pm * (i0 % (int64_t)N)) % (int64_t)N);
                dd[j] = 4u * (uint32_t)((8 * pm) % (int64_t)N);
                rot[j] = tw_table(dd[j], N, thi, tlo);  // W^(8p)
            }
            for (int kb = w.kb0; kb < w.kb1; ++kb) {
                if (!(ok = mbar_wait(&empty[stage], phase ^ 1u, s_abort, err))) break;
                const uint32_t a_st = a_base + stage * T::kABytes;
                const bool seed = ((kb - w.kb0) % kReseed) == 0;
                uint4 vre[PPT], vim[PPT];
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    if (seed) wv[j] = tw_table(uu[j], N, thi, tlo);
                    gen_pair_w(uu[j], N, wv[j], vre[j], vim[j]);
                    wv[j] = cmul_f2(wv[j], rot[j]);
                    uu[j] += dd[j];
                    if (uu[j] >= 4u * N) uu[j] -= 4u * N;
                }
#pragma unroll
                for (int j = 0; j < PPT; ++j) store_pair(a_st, pg + 32 * j, t, vre[j], vim[j]);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[stage]);
                if (++stage == STG) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
    } else if constexpr (ADJ == 1 && PAIR) {
        // ---------------- paired adjoint epilogue ----------------
        // Lane 32 quarter + lane of row half h holds sample i = i_lo + 128 h +
        // 32 quarter + lane, and TMEM columns 2 c, 2 c + 1 of the half hold
        // Re, Im of G_l[i] for the tile's lag c; each lane adds
        // conj(sigma(c_l[i])) G_l[i] over the lags in order.  The weights depend
        // on i - l only: per half each warp stages the 32 + 127 it needs.
        const int quarter = warp & 3;
        float2 *wts = reinterpret_cast<float2 *>(smem + T::kSmemStage + 8192 * quarter);
        uint32_t chain = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            const Work w = decode(u, single, probs, units);
            const int N = w.P.N;
            const int64_t i_lo = (int64_t)w.mt * 256;  // first sample of the tile
            const int lag_lo = w.nt * (TN / 2);        // first lag of the tile
            const int nl = w.P.ncols / 2;              // lags of the call
            float2 acc[MH];
#pragma unroll
            for (int h = 0; h < MH; ++h) acc[h] = make_float2(0.f, 0.f);
            for (int c0 = w.kb0; c0 < w.kb1; c0 += chunk, ++chain) {
                const uint32_t buf = chain % NB, tpar = (chain / NB) & 1u;
                if (!(ok = mbar_wait(&tmem_full[buf], tpar, s_abort, err))) break;
                tc_fence_after();
#pragma unroll
                for (int h = 0; h < MH; ++h) {
                    const int64_t i0w = i_lo + 128 * h + 32 * quarter;  // the warp's first sample
                    // wts[k] = sigma(c) at i - l = i0w - (lag0 + lag_lo) - 127 + k
                    const int64_t d0 = i0w - ((int64_t)w.P.lag0 + lag_lo) - (TN / 2 - 1);
                    __syncwarp();
                    for (int k = lane; k < 32 + TN / 2 - 1; k += 32) {
                        int64_t jj = d0 + k;
                        float2 wv = make_float2(0.f, 0.f);
                        if (w.P.flags & NDFT_F_CIRCULAR_LAG) {
                            jj %= N;
                            if (jj < 0) jj += N;
                        }
                        if (jj >= 0 && jj < N) {
                            const float2 r = w.P.sref[jj];
                            const float cr = (r.x > 0.f) ? 1.f : (r.x < 0.f ? -1.f : 0.f);
                            const float cq = (r.y > 0.f) ? 1.f : (r.y < 0.f ? -1.f : 0.f);
                            wv = make_float2(cr, (w.P.flags & NDFT_F_NO_CONJ_REF) ? cq : -cq);  // sigma(c)
                        }
                        wts[k] = wv;
                    }
                    __syncwarp();
#pragma unroll 1
                    for (int g = 0; g < TN / 16; ++g) {
                        uint32_t r[16];
                        tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)((buf + h) * TN + g * 16), r);
                        tmem_wait_ld();
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int cl = g * 8 + q;  // lag within the tile
                            if (lag_lo + cl < nl) {
                                const float gr = __uint_as_float(r[2 * q]), gi = __uint_as_float(r[2 * q + 1]);
                                const float2 wv = wts[lane - cl + (TN / 2 - 1)];
                                acc[h].x = fmaf(wv.x, gr, acc[h].x);
                                acc[h].x = fmaf(wv.y, gi, acc[h].x);
                                acc[h].y = fmaf(wv.x, gi, acc[h].y);
                                acc[h].y = fmaf(-wv.y, gr, acc[h].y);
                            }
                        }
                    }
                    if (MH == 2 && h == 0) {  // half 0 read: its next chain may start
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(tmem_half0);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tmem_empty[buf]);
            }
            if (!ok) break;
            // partial slice (n-tile, split) of the [slices][2N] partials
            float2 *slice = reinterpret_cast<float2 *>(out_base) + (int64_t)(w.nt * w.P.nsplit + w.split) * N;
#pragma unroll
            for (int h = 0; h < MH; ++h) {
                const int64_t i = i_lo + 128 * h + 32 * quarter + lane;
                if (i < N) slice[i] = acc[h];
            }
        }
    } else if constexpr (ADJ == 1) {
        // ---------------- adjoint epilogue ----------------
        // Row r = 2 i + c of the tile holds component c of G_l[i] for the tile's
        // 256 lags.  Lanes 2k and 2k + 1 of a warp hold the two components of one
        // sample, so each lane gets its partner's value by a shuffle and adds
        //   c = 0: sr G_r + si G_i,   c = 1: sr G_i - si G_r
        // (conj(sigma(c_l[i])) G_l[i], sigma(c_l[i]) = (sr, si)) over the lags in
        // order; the unit's per-row sums go to its slice of the partials.  The
        // weights depend on i - l only: for each row half each warp stages the
        // 16 + 255 it needs in its own 4 KB of shared memory (warp-level
        // synchronisation only, so a warp that gives up on a wait cannot leave
        // another one blocked).
        const int quarter = warp & 3;
        float2 *wts = reinterpret_cast<float2 *>(smem + T::kSmemStage + 4096 * quarter);
        uint32_t chain = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            const Work w = decode(u, single, probs, units);
            const int N = w.P.N;
            const int i_lo = w.mt * (T::kRows / 2);  // first sample of the tile
            const int col_lo = w.nt * TN;             // first lag column of the tile
            float acc[MH];
#pragma unroll
            for (int h = 0; h < MH; ++h) acc[h] = 0.f;
            const float csign = (lane & 1) ? -1.f : 1.f;
            for (int c0 = w.kb0; c0 < w.kb1; c0 += chunk, ++chain) {
                const uint32_t buf = chain % NB, tpar = (chain / NB) & 1u;
                if (!(ok = mbar_wait(&tmem_full[buf], tpar, s_abort, err))) break;
                tc_fence_after();
#pragma unroll
                for (int h = 0; h < MH; ++h) {
                    const int il0 = 64 * h + 16 * quarter;  // the warp's first sample in the tile
                    const int il = il0 + (lane >> 1);       // this lane's sample
                    // wts[k] = sigma(c) at i - l = i_lo + il0 - lag0 - col_lo - 255 + k
                    const int64_t d0 = (int64_t)i_lo + il0 - (w.P.lag0 + col_lo) - (TN - 1);
                    __syncwarp();
                    for (int k = lane; k < 16 + TN - 1; k += 32) {
                        int64_t jj = d0 + k;
                        float2 wv = make_float2(0.f, 0.f);
                        if (w.P.flags & NDFT_F_CIRCULAR_LAG) {
                            jj %= N;
                            if (jj < 0) jj += N;
                        }
                        if (jj >= 0 && jj < N) {
                            const float2 r = w.P.sref[jj];
                            const float cr = (r.x > 0.f) ? 1.f : (r.x < 0.f ? -1.f : 0.f);
                            const float cq = (r.y > 0.f) ? 1.f : (r.y < 0.f ? -1.f : 0.f);
                            wv = make_float2(cr, (w.P.flags & NDFT_F_NO_CONJ_REF) ? cq : -cq);  // sigma(c)
                        }
                        wts[k] = wv;
                    }
                    __syncwarp();
#pragma unroll 1
                    for (int g = 0; g < TN / 16; ++g) {
                        uint32_t r[16];
                        tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)((buf + h) * TN + g * 16), r);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float v = __uint_as_float(r[j]);
                            const float o = __shfl_xor_sync(0xffffffffu, v, 1);
                            const int cl = g * 16 + j;  // lag column within the tile
                            if (col_lo + cl < w.P.ncols) {
                                const float2 wv = wts[(il - il0) - cl + (TN - 1)];
                                acc[h] = fmaf(wv.x, v, acc[h]);
                                acc[h] = fmaf(csign * wv.y, o, acc[h]);
                            }
                        }
                    }
                    if (MH == 2 && h == 0) {  // half 0 read: its next chain may start
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(tmem_half0);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tmem_empty[buf]);
            }
            if (!ok) break;
            // partial slice (n-tile, split) of the [slices][2N] partials
            const int64_t slice = (int64_t)(w.nt * w.P.nsplit + w.split) * 2LL * N;
#pragma unroll
            for (int h = 0; h < MH; ++h) {
                const int64_t row = (int64_t)w.mt * T::kRows + 128 * h + 32 * quarter + lane;
                if (row < 2LL * N) out_base[slice + row] = acc[h];
            }
        }
    } else {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3;
        uint32_t chain = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            const Work w = decode(u, single, probs, units);
            // output rows: G of the adjoint (two per sample, or one per sample paired), or bins
            const int64_t limit_m = ADJ == 2 ? (PAIR ? (int64_t)w.P.N : 2LL * w.P.N) : 2LL * w.P.nbins;
            for (int c0 = w.kb0; c0 < w.kb1; c0 += chunk, ++chain) {
                const uint32_t buf = chain % NB, tpar = (chain / NB) & 1u;
                if (!(ok = mbar_wait(&tmem_full[buf], tpar, s_abort, err))) break;
                tc_fence_after();
                // the first chain of a unit stores; later chains are added in L2 with
                // fire-and-forget reductions (round to nearest).  Each address is
                // written by one thread only, in chain order, so the sum is
                // deterministic.
                const bool first = (c0 == w.kb0);
                if (PAIR && out_tma) {
                    // Paired tile: 32-column groups, each two tcgen05.ld of 16
                    // columns -> one of two 4 KB staging buffers [32 cols][32 rows]
                    // -> one bulk tensor store / add (box 32 x 32) by lane 0.  As
                    // below, lane 0 waits for all of the previous chain's copies
                    // before the chain's first copy (adds land in chain order) and,
                    // before refilling a buffer, for the copy issued two groups
                    // earlier to have read it.
                    const uint32_t wst = smem_u32(smem + T::kSmemStage) + (uint32_t)quarter * 8192u;
                    const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
                    const int mrow0 = w.mt * T::kRows + 32 * quarter;
                    constexpr int GPH = TN / 32;  // groups per row half
                    constexpr int NG = MH * GPH;
#pragma unroll 1
                    for (int g = 0; g < NG; ++g) {
                        const uint32_t tc = (uint32_t)((buf + g / GPH) * TN + (g % GPH) * 32);
                        uint32_t ra[16], rb[16];
                        tmem_ld16(trow + tc, ra);
                        tmem_ld16(trow + tc + 16, rb);
                        tmem_wait_ld();
                        if (MH == 2 && g + 1 == GPH) {  // every load of half 0 has completed
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(tmem_half0);
                        }
                        if (g + 1 == NG) {  // the whole accumulator has been read
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&tmem_empty[buf]);
                        }
                        const uint32_t sb = wst + (uint32_t)(g & 1) * 4096u;
                        if (lane == 0) {
                            if (g == 0) bulk_wait_all();
                            else if (g > 1) bulk_wait_read1();
                        }
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            asm volatile("st.shared.b32 [%0], %1;" ::"r"(sb + (uint32_t)(j * 32 + lane) * 4u), "r"(ra[j])
                                         : "memory");
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            asm volatile("st.shared.b32 [%0], %1;" ::"r"(sb + (uint32_t)((16 + j) * 32 + lane) * 4u),
                                         "r"(rb[j])
                                         : "memory");
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) {
                            const int mrow = mrow0 + 128 * (g / GPH);
                            const int col = w.nt * TN + (g % GPH) * 32;
                            if (first) tma_store_out(&omap, sb, mrow, col, w.split);
                            else tma_reduce_out(&omap, sb, mrow, col, w.split);
                            bulk_commit();
                        }
                    }
                    continue;
                }
                if (out_tma) {
                    // Each epilogue warp drains its own 32 TMEM lanes (rows) on its own:
                    // 16-column groups go TMEM -> registers -> one of two 2 KB staging
                    // buffers [16 cols][32 rows] -> one bulk tensor store (first chain)
                    // or add (later chains) issued by lane 0.  The next group's TMEM
                    // load is in flight while the current one is staged, and a buffer
                    // is refilled once the bulk copy issued two groups earlier has read
                    // it.  Lane 0 waits for all of its previous chain's copies before
                    // the first copy of a chain, so the additions to each row land in
                    // chain order (deterministic sums).  TMEM is released as soon as
                    // the warp's last load has completed.
                    const uint32_t wst = smem_u32(smem + T::kSmemStage) + (uint32_t)quarter * 4096u;
                    const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
                    const int mrow0 = w.mt * T::kRows + 32 * quarter;
                    constexpr int GPH = TN / 16;       // 16-column groups per row half
                    constexpr int NG = MH * GPH;       // groups per chain (even)
                    auto tcol = [&](int g) { return (uint32_t)((buf + g / GPH) * TN + (g % GPH) * 16); };
                    // bulk copy c of the chain uses buffer c & 1 (without partial groups
                    // every group is one copy, so c = g)
                    int ncopy = 0;
                    auto drain = [&](const uint32_t (&r)[16], int g) {
                        const int cidx = BT ? ncopy : g;
                        const uint32_t sb = wst + (uint32_t)(cidx & 1) * 2048u;
                        const int colg = w.nt * TN + (g % GPH) * 16;  // the group's first column
                        if (BT && w.P.ncols - colg < 16) {
                            if (lane == 0 && g == 0) bulk_wait_all();
                            // batched: the map spans all problems, so a group that runs past
                            // this problem's last column is written element by element
                            const int valid = w.P.ncols - colg;
                            const int64_t m = mrow0 + 128 * (g / GPH) + lane;
                            if (valid > 0 && m < limit_m) {
                                float *dst = out_base + w.out_off + (int64_t)colg * w.P.ld + m;
#pragma unroll
                                for (int j = 0; j < 16; ++j) {
                                    if (j >= valid) break;
                                    if (first) dst[j * w.P.ld] = __uint_as_float(r[j]);
                                    else red_add_f32(dst + j * w.P.ld, __uint_as_float(r[j]));
                                }
                            }
                            return;
                        }
                        if (lane == 0) {
                            if (g == 0) bulk_wait_all();  // the previous chain's copies are complete
                            else if (cidx > 0) bulk_wait_read1();  // copy cidx - 2 has read this buffer
                        }
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            asm volatile("st.shared.b32 [%0], %1;" ::"r"(sb + (uint32_t)(j * 32 + lane) * 4u), "r"(r[j])
                                         : "memory");
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) {
                            const int mrow = mrow0 + 128 * (g / GPH);
                            const int col = (BT ? w.P.crow0 : 0) + colg;
                            if (first) tma_store_out(&omap, sb, mrow, col, w.split);
                            else tma_reduce_out(&omap, sb, mrow, col, w.split);
                            bulk_commit();
                        }
                        if (BT) ++ncopy;
                    };
                    uint32_t ra[16], rb[16];
                    tmem_ld16(trow + tcol(0), ra);
                    tmem_wait_ld();
#pragma unroll 1
                    for (int g = 0; g < NG; g += 2) {
                        tmem_ld16(trow + tcol(g + 1), rb);
                        drain(ra, g);
                        tmem_wait_ld();
                        if (MH == 2 && g + 2 == GPH) {  // every load of half 0 has completed
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(tmem_half0);
                        }
                        const bool more = g + 2 < NG;
                        if (more) {
                            tmem_ld16(trow + tcol(g + 2), ra);
                        } else {
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&tmem_empty[buf]);
                        }
                        drain(rb, g + 1);
                        if (more) tmem_wait_ld();
                    }
                    continue;
                }
#pragma unroll 1
                for (int h = 0; h < MH; ++h) {
                    const int64_t m = (int64_t)w.mt * T::kRows + 128 * h + 32 * quarter + lane;
#pragma unroll 1
                    for (int cc = 0; cc < TN; cc += 32) {
                        uint32_t r[32];
                        tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)((buf + h) * TN + cc), r);
                        tmem_wait_ld();
                        const int64_t col0 = (int64_t)w.nt * TN + cc;
                        if (m < limit_m && ndft_in(w.P.ld >= limit_m, err)) {
                            float *dst = out_base + w.out_off + col0 * w.P.ld + m;
                            const int64_t left = w.P.ncols - col0;
                            const int nj = left < 32 ? (int)left : 32;
                            if (first) {
#pragma unroll
                                for (int j = 0; j < 32; ++j)
                                    if (j < nj) dst[j * w.P.ld] = __uint_as_float(r[j]);
                            } else {
#pragma unroll
                                for (int j = 0; j < 32; ++j)
                                    if (j < nj) red_add_f32(dst + j * w.P.ld, __uint_as_float(r[j]));
                            }
                        }
                    }
                    if (MH == 2 && h == 0) {  // half 0 read: its next chain may start
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(tmem_half0);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tmem_empty[buf]);
            }
        }
        if (out_tma && lane == 0) bulk_wait_all();  // this warp's bulk copies done before exit
    }

    __syncthreads();
    if (*s_abort) {
        // give any copy or MMA still in flight time to land before the memory goes away
        const long long t0 = clock64();
        while (clock64() - t0 < 200000) {
        }
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// ---- the 2-SM tile (tcgen05 cta_group::2) ---------------------------------------------
// A CTA pair computes one 256 x 256 tile with M = 256 MMAs issued by the even
// CTA: each CTA generates its own 128 rows of A and loads its own 128 columns
// of B into the same shared-memory offsets, and each CTA's tensor memory holds
// its 128 rows of the accumulator.  A stage is then 32 KiB per CTA (half of
// the 256-row tile's 64 KiB), so six stages fit, and the 256 accumulator
// columns per chain leave room for two accumulators used in turn: the fold-out
// of one chain overlaps the MMAs of the next.
//   full[s]       (even CTA) 1 arrival with 32 KiB expected (its TMA thread),
//                 16 KiB from each CTA's TMA, and 8 producer warps of each CTA
//   empty[s]      (both) one MMA commit, multicast to the pair
//   tmem_full[b]  (both) one MMA commit, multicast to the pair
//   tmem_empty[b] (even CTA) the 4 epilogue warps of each CTA
// Arrivals on the even CTA's barriers from the odd CTA are remote
// (shared::cluster addresses from mapa).
namespace pair2 {
constexpr int kStages = 6;
constexpr int kABytes = 128 * 128;  // 128 rows x 64 K bf16
constexpr int kBBytes = 128 * 128;  // 128 columns x 64 K bf16
constexpr size_t kSmemA = 0;
constexpr size_t kSmemB = kSmemA + (size_t)kStages * kABytes;
constexpr size_t kSmemTab = kSmemB + (size_t)kStages * kBBytes;
constexpr size_t kSmemStage = (kSmemTab + (size_t)(kMaxThi + R_LO) * sizeof(float2) + 127) / 128 * 128;
constexpr size_t kSmemBar = kSmemStage + 4 * 4096;
constexpr size_t kSmemTotal = kSmemBar + 256 + 1024;
static_assert(kSmemTotal <= 232448, "shared memory of one CTA");
// kind::f16, D fp32, A/B bf16, both K-major, N = 256, M = 256 (the pair)
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(256 >> 4) << 24);

__device__ __forceinline__ uint32_t peer_addr(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
// arrival on the even CTA's barrier with the default (release, CTA-scope)
// semantics; a cluster-scope release here costs a fence per arrival (it made the
// whole pipeline about 2x slower)
__device__ __forceinline__ void arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// TMA load of this CTA's B half, completion signalled on the even CTA's barrier
__device__ __forceinline__ void tma_load_b_pair(uint32_t dst, const CUtensorMap *map, int32_t row, uint32_t bar_cl) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(bar_cl)
        : "memory");
}
__device__ __forceinline__ void umma2(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void commit2_mc(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)0x3)
        : "memory");
}
}  // namespace pair2

// `tmap` has a 128-row box (one CTA's B half).  Forward single-surface
// contraction only (the batched and adjoint modes keep the one-CTA tile).
// ATAB: the conjugate-paired contraction with its A operand from the plan's
// table (`amap`, 128-row box: each CTA loads its 128 rows, completion on the
// even CTA's barrier like B); no A producer warps run.
// BM = kBForm (with ATAB): the B operand is not loaded but formed in shared
// memory by 16 producer warps of each CTA from the inputs (`bg`), the same
// chunks the packing kernel writes: thread g of a CTA forms chunk t = g & 7 of
// the CTA's lag column j = g >> 3 (rows 2 j, 2 j + 1 of its 128-row half).
// The m-tile-0 units also sum v + sigma(v) of their columns over their K range
// into bg.dc[split][col] (bin 0), in a fixed order.
// BM = kBAhead (with ATAB): B is packed just in time by the tile's own warps.
// An item is 16 K blocks x 64 lag columns, the B half one CTA loads for one
// unit; the four units of a column tile (its m-tiles, on four pairs of the
// same wave) load the same items.  16 packer warps per CTA walk the CTA's own
// item sequence at most bg.look items ahead of its TMA thread, claim each
// item that no other CTA has claimed (atomicCAS on its state), write it into
// the packed buffer exactly as k_pack_pair does (bin-0 sums per item) and
// release it (gpu-scope fence, state 2); the TMA thread waits for state 2
// (acquire, then a proxy fence) before loading it, so the B tile is read from
// L2 by the CTAs that share it moments after it was written.  A claimed item
// is packed without waiting on anything, and a CTA's packers wait only for
// their own CTA's TMA thread, which waits only for claimed items or for items
// its own packers will reach: no CTA waits for one that is not resident.
__host__ __device__ constexpr int pair_gen_warps(int bm) { return bm != kBTma ? 16 : kGenWarps; }
__host__ __device__ constexpr int pair_threads(int bm) { return (2 + pair_gen_warps(bm) + 4) * 32; }

// 16-byte global store with an L2 cache policy.
__device__ __forceinline__ void st_keep(uint4 *p, const uint4 &v, uint64_t policy) {
    asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w), "l"(policy)
                 : "memory");
}

// Bounded wait until *f >= target (acquire at gpu scope).
__device__ __forceinline__ bool flag_wait(const int32_t *f, int32_t target, volatile int32_t *abort_flag,
                                          int32_t *err) {
    const long long t0 = clock64();
    for (;;) {
        int32_t v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
        if (v >= target) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            dev_set_error(err, kDevTimeout);
            return false;
        }
        __nanosleep(32);
    }
}

template <bool ATAB, int BM>
__global__ void __launch_bounds__(pair_threads(BM), 1)
    k_ternary_gemm_pair(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap omap,
                        int out_tma, Problem single, int64_t nunits, int chunk, int starve, float *__restrict__ out_base,
                        int32_t *err, const __grid_constant__ CUtensorMap amap, const BGen bg) {
    static_assert(ATAB || BM == kBTma, "operand generation goes with the A table");
    constexpr bool BGEN = BM == kBForm;
    using namespace pair2;
    const uint32_t rank = cluster_rank();
    const bool lead = rank == 0;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    float2 *s_thi = reinterpret_cast<float2 *>(smem + kSmemTab);
    float2 *s_tlo = s_thi + kMaxThi;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kSmemBar);
    uint64_t *empty = full + kStages;
    uint64_t *tmem_full = empty + kStages;  // [2]
    uint64_t *tmem_empty = tmem_full + 2;   // [2]
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(tmem_empty + 2);
    volatile int32_t *s_abort = reinterpret_cast<volatile int32_t *>(s_tmem + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t a_base = smem_u32(smem + kSmemA), b_base = smem_u32(smem + kSmemB);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], (ATAB && !BGEN) ? 1 : 1 + 2 * pair_gen_warps(BM));
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tmem_full[b], 1);
            mbar_init(&tmem_empty[b], 8);
        }
        *s_abort = 0;
        s_tmem[3] = 0;  // kBAhead: the TMA thread's position in its item sequence
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
    }
    if (warp == 1) {
        // one warp of each CTA of the pair allocates, collectively
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // both CTAs' barriers are initialised before any remote arrival
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp == 0) {
        // ---------------- TMA producer (each CTA its B half) ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            bool started = false;  // kBAhead: past the first position of the item sequence
            volatile int32_t *s_prog = reinterpret_cast<volatile int32_t *>(s_tmem + 3);
            for (int64_t u = blockIdx.x / 2; u < nunits && ok; u += gridDim.x / 2) {
                const Work w = decode(u, single, nullptr, nullptr);
                for (int kb = w.kb0; kb < w.kb1; ++kb) {
                    if (!(ok = mbar_wait(&empty[stage], phase ^ 1u, s_abort, err))) break;
                    if (starve) continue;
                    if (lead) mbar_arrive_tx(&full[stage], (BGEN ? 0 : 2 * kBBytes) + (ATAB ? 2 * kABytes : 0));
                    if constexpr (ATAB) {
                        const int64_t arow = (int64_t)kb * w.P.a_ld + (int64_t)w.mt * 256 + rank * 128;
                        tma_load_b_pair(a_base + stage * kABytes, &amap, (int32_t)arow,
                                        peer_addr(smem_u32(&full[stage]), 0u));
                    }
                    if constexpr (BM == kBAhead) {
                        if ((kb - w.kb0) % 16 == 0) {
                            // the first K block of the next position of this CTA's item
                            // sequence (the packers walk the same one): column block
                            // cx = 2 nt + rank of item (split, j)
                            if (started) *s_prog = *s_prog + 1;
                            started = true;
                            const int64_t item =
                                ((int64_t)w.split * bg.jmax + (kb - w.kb0) / 16) * bg.ncx + 2 * w.nt + (int)rank;
                            if (!(ok = flag_wait(bg.ctr + 1 + item, 2, s_abort, err))) break;
                            asm volatile("fence.proxy.async.global;" ::: "memory");
                        }
                    }
                    if constexpr (!BGEN) {
                        const int64_t row =
                            w.P.b_row0 + (int64_t)kb * w.P.ncols + (int64_t)w.nt * TN + rank * (TN / 2);
                        tma_load_b_pair(b_base + stage * kBBytes, &tmap, (int32_t)row,
                                        peer_addr(smem_u32(&full[stage]), 0u));
                    }
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (even CTA) ----------------
        if (lead && lane == 0) {
            int stage = 0;
            uint32_t phase = 0, chain = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x / 2; u < nunits && ok; u += gridDim.x / 2) {
                const Work w = decode(u, single, nullptr, nullptr);
                for (int c0 = w.kb0; c0 < w.kb1 && ok; c0 += chunk, ++chain) {
                    const int c1 = min(c0 + chunk, w.kb1);
                    const uint32_t buf = chain & 1u, tpar = (chain >> 1) & 1u;
                    if (!(ok = mbar_wait(&tmem_empty[buf], tpar ^ 1u, s_abort, err))) break;
                    tc_fence_after();
                    const uint32_t d0 = tmem + buf * (uint32_t)TN;
                    for (int kb = c0; kb < c1; ++kb) {
                        if (!(ok = mbar_wait(&full[stage], phase, s_abort, err))) break;
                        tc_fence_after();
                        const uint32_t a_st = a_base + stage * kABytes, b_st = b_base + stage * kBBytes;
#pragma unroll
                        for (int k = 0; k < KB / 16; ++k)
                            umma2(d0, umma_desc(a_st + k * 32), umma_desc(b_st + k * 32), (kb > c0 || k > 0) ? 1u : 0u);
                        commit2_mc(&empty[stage]);
                        if (++stage == kStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    commit2_mc(&tmem_full[buf]);
                }
            }
        }
        __syncwarp();
    } else if (warp < 2 + pair_gen_warps(BM)) {
        if constexpr (BM == kBAhead) {
        // ---------------- packers: this CTA's own B items, just ahead of its TMA loads ----------------
        const int g = threadIdx.x - 64;  // 0..511
        const int t = g & 7, lc = g >> 3;
        const PackProb &pp = bg.pp;
        const int N = pp.N;
        const bool caf = bg.caf != 0, conj = !(bg.flags & NDFT_F_NO_CONJ_REF),
                   circ = (bg.flags & NDFT_F_CIRCULAR_LAG) != 0;
        const float2 *r = bg.r + pp.r_off;
        const int64_t ncols2 = 2LL * pp.ncols;
        volatile int32_t *s_cmd = reinterpret_cast<volatile int32_t *>(s_tmem + 2);
        volatile int32_t *s_prog = reinterpret_cast<volatile int32_t *>(s_tmem + 3);
        int32_t q = 0;  // position in this CTA's item sequence
        // B goes to L2 with evict-last priority: the four CTAs that load an item
        // read it moments later (measured: 0.16 GB less DRAM read per launch)
        uint64_t keep;
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
        bool run = true;
        for (int64_t u = blockIdx.x / 2; u < nunits && run; u += gridDim.x / 2) {
            const Work w = decode(u, single, nullptr, nullptr);
            const int cx = 2 * w.nt + (int)rank;
            for (int k0 = w.kb0; k0 < w.kb1; k0 += 16, ++q) {
                const int jb = (k0 - w.kb0) / 16, k1 = min(k0 + 16, w.kb1);
                const int64_t item = ((int64_t)w.split * bg.jmax + jb) * bg.ncx + cx;
                if (g == 0) {
                    // at most bg.look items ahead of the TMA thread; then claim the item
                    // unless another CTA of its column tile has
                    int32_t cmd = 0;
                    const long long t0 = clock64();
                    while (*s_prog < q - bg.look) {
                        if (*s_abort || clock64() - t0 > kWaitCycles) {
                            cmd = -1;
                            break;
                        }
                        __nanosleep(64);
                    }
                    if (cmd == 0) cmd = atomicCAS(bg.ctr + 1 + item, 0, 1) == 0 ? 1 : 0;
                    *s_cmd = cmd;
                }
                gen_bar_n<16>();
                const int32_t cmd = *s_cmd;
                gen_bar_n<16>();  // every packer has read the command before thread 0 writes the next
                if (cmd < 0) {
                    run = false;
                    break;
                }
                if (cmd == 0) continue;
                const int64_t col = (int64_t)cx * 64 + lc;
                const bool live = col < pp.ncols;
                const int64_t lag = (int64_t)pp.lag0 + col;
                const float2 *a = bg.a + pp.a_off + (caf || !live ? 0 : col * pp.ldx);
                const bool vec = (reinterpret_cast<uintptr_t>(a) & 15u) == 0;
                float dsr = 0.f, dsi = 0.f;
                if (live) {
                    for (int kb = k0; kb < k1; ++kb) {
                        float2 v0, v1;
                        pair_samples(a, r, kb * 16 + 2 * t, N, lag, caf, conj, circ, vec, v0, v1);
                        uint4 cre, cim;
                        float dr, di;
                        pair_chunks(v0, v1, cre, cim, dr, di);
                        const int64_t row = (int64_t)kb * ncols2 + 2 * col;
                        st_keep(bg.B + row * 8 + t, cre, keep);
                        st_keep(bg.B + (row + 1) * 8 + t, cim, keep);
                        dsr += dr;
                        dsi += di;
                    }
                }
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    dsr += __shfl_xor_sync(0xffffffffu, dsr, o);
                    dsi += __shfl_xor_sync(0xffffffffu, dsi, o);
                }
                if (t == 0 && live) bg.dc[((int64_t)w.split * bg.jmax + jb) * pp.ncols + col] = make_float2(dsr, dsi);
                // the item's stores, then one release for the CTA's packers (the barrier
                // orders every packer's stores before thread 0's fence)
                asm volatile("fence.proxy.async.global;" ::: "memory");
                gen_bar_n<16>();
                if (g == 0) {
                    __threadfence();
                    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(bg.ctr + 1 + item), "r"(2) : "memory");
                }
            }
        }
        } else if constexpr (BGEN) {
        // ---------------- B producers: this CTA's 64 lag columns (128 rows) ----------------
        const int g = threadIdx.x - 64;  // 0..511
        const int t = g & 7, j0 = g >> 3;  // chunk t of lag column j0 (rows 2 j0, 2 j0 + 1)
        const PackProb &pp = bg.pp;
        const int N = pp.N;
        const bool caf = bg.caf != 0, conj = !(bg.flags & NDFT_F_NO_CONJ_REF),
                   circ = (bg.flags & NDFT_F_CIRCULAR_LAG) != 0;
        const float2 *r = bg.r + pp.r_off;
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x / 2; u < nunits && ok; u += gridDim.x / 2) {
            const Work w = decode(u, single, nullptr, nullptr);
            const bool dcw = w.mt == 0 && bg.dc != nullptr;
            const int64_t col = (int64_t)w.nt * (TN / 2) + rank * (TN / 4) + j0;
            const bool live = col < pp.ncols;
            const int64_t lag = (int64_t)pp.lag0 + col;
            const float2 *a = bg.a + pp.a_off + (caf || !live ? 0 : col * pp.ldx);
            const bool vec = (reinterpret_cast<uintptr_t>(a) & 15u) == 0;
            float dsr = 0.f, dsi = 0.f;
            // inputs of the next K block, loaded while this one is formed and stored
            float2 nv0, nv1, nr0, nr1;
            const float2 zero = make_float2(0.f, 0.f);
            nv0 = nv1 = nr0 = nr1 = zero;
            if (live && w.kb0 < w.kb1) pair_loads(a, r, w.kb0 * 16 + 2 * t, N, lag, caf, circ, vec, nv0, nv1, nr0, nr1);
            for (int kb = w.kb0; kb < w.kb1; ++kb) {
                float2 v0 = nv0, v1 = nv1;
                const float2 r0 = nr0, r1 = nr1;
                if (live && kb + 1 < w.kb1)
                    pair_loads(a, r, (kb + 1) * 16 + 2 * t, N, lag, caf, circ, vec, nv0, nv1, nr0, nr1);
                pair_combine(caf, conj, r0, r1, v0, v1);
                uint4 cre, cim;
                float dr, di;
                pair_chunks(v0, v1, cre, cim, dr, di);
                dsr += dr;
                dsi += di;
                // warp-uniform, so that an abandoned wait leaves no lane behind at the shuffles
                if (!(ok = __all_sync(0xffffffffu, mbar_wait(&empty[stage], phase ^ 1u, s_abort, err)))) break;
                store_pair(b_base + stage * kBBytes, j0, t, cre, cim);
                // the even CTA's MMA reads this CTA's tile through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    if (lead) mbar_arrive(&full[stage]);
                    else arrive_remote(peer_addr(smem_u32(&full[stage]), 0u));
                }
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (!ok || !dcw) continue;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                dsr += __shfl_xor_sync(0xffffffffu, dsr, o);
                dsi += __shfl_xor_sync(0xffffffffu, dsi, o);
            }
            if (t == 0 && live) bg.dc[(int64_t)w.split * pp.ncols + col] = make_float2(dsr, dsi);
        }
        } else if constexpr (!ATAB) {
        // ---------------- A producers: this CTA's 64 bins (128 rows) ----------------
        const int g = threadIdx.x - 64;  // 0..255
        const int t = g & 7, pg = g >> 3;
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x / 2; u < nunits; u += gridDim.x / 2) {
            const Work w = decode(u, single, nullptr, nullptr);
            gen_bar();
            for (int e = g; e < w.P.nth + R_LO; e += kGenWarps * 32) {
                const float2 v = w.P.ang[e];
                if (e < w.P.nth) s_thi[e] = v;
                else s_tlo[e - w.P.nth] = v;
            }
            gen_bar();
            if (!ok) continue;
            const uint32_t N = (uint32_t)w.P.N;
            const uint32_t thi = smem_u32(s_thi), tlo = smem_u32(s_tlo);
            uint32_t uu[2], dd[2];
            float2 wv[2], rot[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int k = w.mt * 128 + (int)rank * 64 + pg + 32 * j;  // bin index
                int64_t pm = ((int64_t)w.P.p0 + k) % (int64_t)N;
                if (pm < 0) pm += N;
                const int64_t i0 = (int64_t)w.kb0 * 8 + t;
                uu[j] = 4u * (uint32_t)((pm * (i0 % (int64_t)N)) % (int64_t)N);
                dd[j] = 4u * (uint32_t)((8 * pm) % (int64_t)N);
                rot[j] = tw_table(dd[j], N, thi, tlo);
            }
            for (int kb = w.kb0; kb < w.kb1; ++kb) {
                if (!(ok = mbar_wait(&empty[stage], phase ^ 1u, s_abort, err))) break;
                const uint32_t a_st = a_base + stage * kABytes;
                const bool seed = ((kb - w.kb0) % kReseed) == 0;
                uint4 vre[2], vim[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    if (seed) wv[j] = tw_table(uu[j], N, thi, tlo);
                    gen_pair_w(uu[j], N, wv[j], vre[j], vim[j]);
                    wv[j] = cmul_f2(wv[j], rot[j]);
                    uu[j] += dd[j];
                    if (uu[j] >= 4u * N) uu[j] -= 4u * N;
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) store_pair(a_st, pg + 32 * j, t, vre[j], vim[j]);
                // the even CTA's MMA reads this CTA's tile through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    if (lead) mbar_arrive(&full[stage]);
                    else arrive_remote(peer_addr(smem_u32(&full[stage]), 0u));
                }
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
        }
    } else {
        // ---------------- epilogue: this CTA's 128 rows ----------------
        const int quarter = warp & 3;
        uint32_t chain = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x / 2; u < nunits && ok; u += gridDim.x / 2) {
            const Work w = decode(u, single, nullptr, nullptr);
            const int64_t limit_m = 2LL * w.P.nbins;
            for (int c0 = w.kb0; c0 < w.kb1; c0 += chunk, ++chain) {
                const uint32_t buf = chain & 1u, tpar = (chain >> 1) & 1u;
                if (!(ok = mbar_wait(&tmem_full[buf], tpar, s_abort, err))) break;
                tc_fence_after();
                const bool first = (c0 == w.kb0);
                const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
                const int mrow = w.mt * 256 + (int)rank * 128 + 32 * quarter;
                auto release = [&]() {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (lead) mbar_arrive(&tmem_empty[buf]);
                        else arrive_remote(peer_addr(smem_u32(&tmem_empty[buf]), 0u));
                    }
                };
                if (out_tma) {
                    // as the one-CTA epilogue: 16-column groups through two 2 KB staging
                    // buffers to bulk tensor stores (first chain) or adds (later chains),
                    // every address receiving its chain sums in order
                    const uint32_t wst = smem_u32(smem + kSmemStage) + (uint32_t)quarter * 4096u;
                    constexpr int NG = TN / 16;
                    auto drain = [&](const uint32_t (&r)[16], int g) {
                        const uint32_t sb = wst + (uint32_t)(g & 1) * 2048u;
                        if (lane == 0) {
                            if (g == 0) bulk_wait_all();
                            else bulk_wait_read1();
                        }
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            asm volatile("st.shared.b32 [%0], %1;" ::"r"(sb + (uint32_t)(j * 32 + lane) * 4u), "r"(r[j])
                                         : "memory");
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) {
                            const int col = w.nt * TN + g * 16;
                            if (first) tma_store_out(&omap, sb, mrow, col, w.split);
                            else tma_reduce_out(&omap, sb, mrow, col, w.split);
                            bulk_commit();
                        }
                    };
                    uint32_t ra[16], rb[16];
                    const uint32_t tc0 = trow + buf * (uint32_t)TN;
                    tmem_ld16(tc0, ra);
                    tmem_wait_ld();
#pragma unroll 1
                    for (int g = 0; g < NG; g += 2) {
                        tmem_ld16(tc0 + (uint32_t)(g + 1) * 16u, rb);
                        drain(ra, g);
                        tmem_wait_ld();
                        const bool more = g + 2 < NG;
                        if (more) tmem_ld16(tc0 + (uint32_t)(g + 2) * 16u, ra);
                        else release();
                        drain(rb, g + 1);
                        if (more) tmem_wait_ld();
                    }
                    continue;
                }
                const int64_t m = (int64_t)mrow + lane;
#pragma unroll 1
                for (int cc = 0; cc < TN; cc += 32) {
                    uint32_t r[32];
                    tmem_ld32(trow + buf * (uint32_t)TN + (uint32_t)cc, r);
                    tmem_wait_ld();
                    const int64_t col0 = (int64_t)w.nt * TN + cc;
                    if (m < limit_m) {
                        float *dst = out_base + w.out_off + col0 * w.P.ld + m;
                        const int64_t left = w.P.ncols - col0;
                        const int nj = left < 32 ? (int)left : 32;
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < nj) {
                                if (first) dst[j * w.P.ld] = __uint_as_float(r[j]);
                                else red_add_f32(dst + j * w.P.ld, __uint_as_float(r[j]));
                            }
                    }
                }
                release();
            }
        }
        if (out_tma && lane == 0) bulk_wait_all();
    }

    __syncthreads();
    if (*s_abort) {
        const long long t0 = clock64();
        while (clock64() - t0 < 200000) {
        }
    }
    // neither CTA leaves while the pair's MMAs may still use its shared or tensor memory
    cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// ---- packing of the B operand ------------------------------------------------------
// Row (kb, col) of the packed buffer holds samples i = 8 kb .. 8 kb + 7 of column
// col, 16 bytes each: [v_hi_r, v_lo_r, v_hi_i, v_lo_i, s_r, s_r, s_i, s_i] (bf16).
__device__ __forceinline__ uint4 pack_entry(float2 v) {
    const __nv_bfloat162 hi = __floats2bfloat162_rn(v.x, v.y);
    const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x - __low2float(hi), v.y - __high2float(hi));
    const uint32_t uh = *reinterpret_cast<const uint32_t *>(&hi);
    const uint32_t ul = *reinterpret_cast<const uint32_t *>(&lo);
    const uint32_t sr = (v.x > 0.f) ? 0x3F803F80u : ((v.x < 0.f) ? 0xBF80BF80u : 0u);
    const uint32_t si = (v.y > 0.f) ? 0x3F803F80u : ((v.y < 0.f) ? 0xBF80BF80u : 0u);
    return make_uint4(__byte_perm(uh, ul, 0x5410), __byte_perm(uh, ul, 0x7632), sr, si);
}


__device__ __forceinline__ float2 lag_product(const PackProb &P, const float2 *__restrict__ a,
                                              const float2 *__restrict__ r, int64_t col, int64_t i, uint32_t flags) {
    int64_t j = i - (P.lag0 + col);
    float2 ref = make_float2(0.f, 0.f);
    if (flags & NDFT_F_CIRCULAR_LAG) {
        j %= P.N;
        if (j < 0) j += P.N;
    }
    if (j >= 0 && j < P.N) {
        ref = r[j];
        if (!(flags & NDFT_F_NO_CONJ_REF)) ref.y = -ref.y;
    }
    return cox_f32(a[i], ref);
}

// Packs nprob problems; thread e handles entry t = e & 7 of row e >> 3 of the
// problem that row falls in (prefix[] holds each problem's first flat row).
__global__ void k_pack(const PackProb *__restrict__ probs, const int64_t *__restrict__ prefix, int nprob,
                       PackProb single, int64_t total_rows, uint32_t flags, bool caf, const float2 *__restrict__ a_base,
                       const float2 *__restrict__ r_base, uint4 *__restrict__ B, int32_t *err) {
    const int64_t total = total_rows * 8;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e & 7);
        const int64_t frow = e >> 3;
        PackProb P = single;
        int64_t local = frow;
        if (probs) {
            int lo = 0, hi = nprob - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (prefix[mid] <= frow) lo = mid;
                else hi = mid - 1;
            }
            P = probs[lo];
            local = frow - prefix[lo];
        }
        // rows of one problem number < 2^31 (checked at plan time): 32-bit division
        const uint32_t kb = (uint32_t)local / (uint32_t)P.ncols;
        const uint32_t col = (uint32_t)local - kb * (uint32_t)P.ncols;
        const int64_t i = (int64_t)kb * 8 + t;
        float2 v = make_float2(0.f, 0.f);
        const float2 *a = a_base + P.a_off;
        if (i < P.N) v = caf ? lag_product(P, a, r_base + P.r_off, col, i, flags) : a[col * P.ldx + i];
        if (ndft_in(local < (int64_t)P.kblocks * P.ncols, err)) B[(P.row0 + local) * 8 + t] = pack_entry(v);
    }
}

// One problem: block (x, y) packs columns [32 x, 32 x + 32) of K blocks
// [8 y', 8 y' + 8) for y' = y, y + gridDim.y, ... < gy, one 16-byte entry per
// thread and K block, no division: one tile per block on a full grid, or a
// grid bounded in y that leaves room on every SM for a contraction CTA.
constexpr int kPackKb = 8;
__global__ void __launch_bounds__(256) k_pack_single(PackProb P, uint32_t flags, bool caf,
                                                     const float2 *__restrict__ a_base,
                                                     const float2 *__restrict__ r_base, uint4 *__restrict__ B,
                                                     int gy, int32_t *err) {
    const int t = threadIdx.x & 7;
    const int col = blockIdx.x * 32 + (threadIdx.x >> 3);
    if (col >= P.ncols) return;
    const float2 *a = a_base + P.a_off;
    const float2 *r = r_base + P.r_off;
    for (int by = blockIdx.y; by < gy; by += gridDim.y) {
        const int kb0 = by * kPackKb;
        const int kb1 = min(kb0 + kPackKb, P.kblocks);
#pragma unroll 2
        for (int kb = kb0; kb < kb1; ++kb) {
            const int64_t i = (int64_t)kb * 8 + t;
            float2 v = make_float2(0.f, 0.f);
            if (i < P.N) v = caf ? lag_product(P, a, r, col, i, flags) : a[(int64_t)col * P.ldx + i];
            if (ndft_in(kb < P.kblocks, err)) B[(P.row0 + (int64_t)kb * P.ncols + col) * 8 + t] = pack_entry(v);
        }
    }
}

// Many problems: tiles of 8 K blocks x 32 columns (the k_pack_single block)
// numbered problem by problem; tile_prefix[c] is problem c's first tile.  Each
// block of a persistent grid packs one contiguous range of tiles: it finds the
// problem of its first tile by a binary search over tile_prefix and then steps
// through the problems in order.
__global__ void __launch_bounds__(256) k_pack_tiles(const PackProb *__restrict__ probs,
                                                    const int64_t *__restrict__ tile_prefix, int nprob,
                                                    uint32_t flags, const float2 *__restrict__ a_base,
                                                    const float2 *__restrict__ r_base, uint4 *__restrict__ B,
                                                    int32_t *err) {
    const int64_t total = tile_prefix[nprob];
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per;
    const int64_t t1 = t0 + per < total ? t0 + per : total;
    const int t = threadIdx.x & 7;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_prefix[mid] <= t0) lo = mid;
        else hi = mid - 1;
    }
    for (int64_t tile = t0; tile < t1; ++tile) {
        while (tile >= tile_prefix[lo + 1]) ++lo;
        const PackProb &P = probs[lo];
        const int ct = (P.ncols + 31) / 32;
        const int local = (int)(tile - tile_prefix[lo]);
        const int kbt = local / ct;
        const int col = (local - kbt * ct) * 32 + (threadIdx.x >> 3);
        if (col >= P.ncols) continue;
        const float2 *a = a_base + P.a_off;
        const float2 *r = r_base + P.r_off;
        const int kb0 = kbt * kPackKb;
        const int kb1 = min(kb0 + kPackKb, P.kblocks);
#pragma unroll 2
        for (int kb = kb0; kb < kb1; ++kb) {
            const int64_t i = (int64_t)kb * 8 + t;
            float2 v = make_float2(0.f, 0.f);
            if (i < P.N) v = lag_product(P, a, r, col, i, flags);
            if (ndft_in(kb < P.kblocks, err)) B[(P.row0 + (int64_t)kb * P.ncols + col) * 8 + t] = pack_entry(v);
        }
    }
}

// Adjoint B operand: row (kb, l) holds bins 16 kb .. 16 kb + 15 of dA[l] as four
// bf16 each, [hi_r, lo_r, hi_i, lo_i] (hi = bf16(a), lo = bf16(a - hi)); bins
// past nbins are zero.  One 8-byte entry per thread, coalesced over the bins.
__global__ void __launch_bounds__(256) k_pack_adjoint(const float2 *__restrict__ dA, int nbins, int nlags,
                                                       int kblocks, uint2 *__restrict__ B) {
    const int64_t total = (int64_t)nlags * kblocks * 16;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = e / ((int64_t)kblocks * 16);
        const int p = (int)(e - l * kblocks * 16);
        const float2 a = p < nbins ? dA[l * nbins + p] : make_float2(0.f, 0.f);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(a.x, a.y);
        const __nv_bfloat162 lo = __floats2bfloat162_rn(a.x - __low2float(hi), a.y - __high2float(hi));
        const uint32_t uh = *reinterpret_cast<const uint32_t *>(&hi);
        const uint32_t ul = *reinterpret_cast<const uint32_t *>(&lo);
        const int kb = p >> 4, k = p & 15;
        B[((int64_t)kb * nlags + l) * 16 + k] = make_uint2(__byte_perm(uh, ul, 0x5410), __byte_perm(uh, ul, 0x7632));
    }
}

// ---- conjugate-paired form: packing and fold --------------------------------------
// With F[-p][i] = conj(F[p][i]) and sigma(conj w) = conj(sigma(w)) (Eq. 8 and
// the sign cases of Eq. 2), bins +c and -c share U = S_r v + F_r sigma(v) and
// V = S_i v + F_i sigma(v) (real matrices times the complex v):
//     X[+c] = U + j V,   X[-c] = U - j V.
// As one real GEMM: row R of frequency c pairs [S_r, S_r, F_hi_r, F_lo_r] and
// row I [S_i, S_i, F_hi_i, F_lo_i] per sample with two B columns per input
// column, (col, r) = [v_hi_r, v_lo_r, s_r, s_r] and (col, i) = [v_hi_i,
// v_lo_i, s_i, s_i]; the four results per (c, col) are
//     a = R.(col, r) = Re U,  d = R.(col, i) = Im U,
//     e = I.(col, r) = Re V,  b = I.(col, i) = Im V,
// so X[+c] = (a - b) + j (d + e) and X[-c] = (a + b) + j (d - e).  Half the
// multiply-adds of the unpaired rows per output bin.  c = 0 (W = 1) needs
// no GEMM row: X[0] = sum_i (v + sigma(v)) is summed by the packing kernel.
//
// B row (kb, 2 col + comp) holds samples 16 kb .. 16 kb + 15 of component comp
// of column col, 4 bf16 each: chunk t (16 bytes) = samples a = 16 kb + 2 t and
// a + 1 as [v_hi(a), v_hi(a+1), v_lo(a), v_lo(a+1), sigma(a), sigma(a+1),
// sigma(a), sigma(a+1)] against the A rows' [S, S, F_hi, F_lo] in the same
// order.  Thread t of a column's 8 packs samples 2 t and
// 2 t + 1 of each K block into both rows and adds v + sigma(v) of them to the
// column's DC sum; the 8 partial sums of a column are combined in a fixed
// order and written per K-block tile (dc[tile][col]).
constexpr int kPairPackKb = 16;  // K blocks (16 samples each) per packing tile


__global__ void __launch_bounds__(256) k_pack_pair(PackProb P, uint32_t flags, bool caf,
                                                   const float2 *__restrict__ a_base,
                                                   const float2 *__restrict__ r_base, uint4 *__restrict__ B,
                                                   float2 *__restrict__ dc, int gy, int32_t *err) {
    const int t = threadIdx.x & 7;
    const int col = blockIdx.x * 32 + (threadIdx.x >> 3);
    const bool live = col < P.ncols;  // whole 8-lane groups are live or not
    const int64_t row_end = P.row0 + (int64_t)P.kblocks * 2 * P.ncols;  // this problem's packed rows
    const float2 *a = a_base + P.a_off + (caf ? 0 : (int64_t)col * P.ldx);
    const float2 *r = r_base + P.r_off;
    const int64_t ncols2 = 2LL * P.ncols;
    const bool conj = !(flags & NDFT_F_NO_CONJ_REF), circ = (flags & NDFT_F_CIRCULAR_LAG) != 0;
    const int N = P.N;
    const int64_t lag = (int64_t)P.lag0 + col;
    const bool vec = (reinterpret_cast<uintptr_t>(a) & 15u) == 0;  // rows of odd length start at 8 bytes
    for (int by = blockIdx.y; by < gy; by += gridDim.y) {
        const int kb0 = by * kPairPackKb;
        const int kb1 = min(kb0 + kPairPackKb, P.kblocks);
        float sr = 0.f, si = 0.f;
        if (live) {
            for (int kb = kb0; kb < kb1; ++kb) {
                const int i = kb * 16 + 2 * t;  // < 2^18 + 16
                float2 v0, v1;
                pair_samples(a, r, i, N, lag, caf, conj, circ, vec, v0, v1);
                const int64_t row = P.row0 + (int64_t)kb * ncols2 + 2LL * col;
                uint4 cre, cim;
                float dr, di;
                pair_chunks(v0, v1, cre, cim, dr, di);
                if (ndft_in(row >= P.row0 && row + 1 < row_end, err)) {
                    B[row * 8 + t] = cre;
                    B[(row + 1) * 8 + t] = cim;
                }
                sr += dr;
                si += di;
            }
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (live && t == 0 && dc && ndft_in(by < gy, err)) dc[(int64_t)by * P.ncols + col] = make_float2(sr, si);
    }
}

// Split-K sum and pair fold into the output [cols][nbins]: block (x, y) =
// output column x, frequencies c = 1 + 256 y .. 256 y + 256, one per thread.
// Slot c - 1 of the partials [split][2 cols][2 S] (rows 2 s, 2 s + 1 = R, I;
// columns 2 col, 2 col + 1 = r, i): each of a, b, d, e summed over the splits
// in order, once, then combined into X[+c] and X[-c], written to the window's
// bins p = c and p = N - c (mod N) that it holds (once where they coincide).
// Bin 0 (c = 0) from the DC tiles, by warp 0 of the y = 0 block.  The split
// loads are issued ahead of the (ordered) additions.  Deterministic.
// With ABS the magnitude |X| (fp32, each operation rounded once) is written.
constexpr int kFoldBins = 256;
__device__ __forceinline__ float cabs_rn(float2 v) {
    return __fsqrt_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)));
}
template <bool ABS>
__global__ void __launch_bounds__(kFoldBins) k_pair_fold(const float *__restrict__ part, int nsplit,
                                                         int64_t split_stride, int S, int N, int p0, int nbins,
                                                         const float2 *__restrict__ dc, int gy, int ncols,
                                                         void *__restrict__ out_v, int32_t *err) {
    const int col = blockIdx.x;
    const int64_t c = 1 + (int64_t)blockIdx.y * kFoldBins + threadIdx.x;
    const int64_t S2 = 2LL * S;
    float2 *o = static_cast<float2 *>(out_v) + (int64_t)col * nbins;
    float *oa = static_cast<float *>(out_v) + (int64_t)col * nbins;
    if (c <= S && ndft_in(col < ncols, err)) {
        // the window positions of bins +c and -c (>= nbins: not in the window)
        int64_t kp = (c - p0) % N, km = (N - c - p0) % N;
        if (kp < 0) kp += N;
        if (km < 0) km += N;
        const bool wp = kp < nbins, wm = km < nbins && km != kp;
        if (wp || wm) {
            const int64_t s = c - 1;
            const float2 *pr = reinterpret_cast<const float2 *>(part + (int64_t)(2 * col) * S2 + 2 * s);      // (a, e)
            const float2 *pi = reinterpret_cast<const float2 *>(part + (int64_t)(2 * col + 1) * S2 + 2 * s);  // (d, b)
            const int64_t st = split_stride / 2;  // float2 elements between splits
            float2 ae = pr[0], db = pi[0];
            int sp = 1;
            for (; sp + 4 <= nsplit; sp += 4) {
                float2 u[4], v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    u[q] = pr[(sp + q) * st];
                    v[q] = pi[(sp + q) * st];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ae.x = __fadd_rn(ae.x, u[q].x);
                    ae.y = __fadd_rn(ae.y, u[q].y);
                    db.x = __fadd_rn(db.x, v[q].x);
                    db.y = __fadd_rn(db.y, v[q].y);
                }
            }
            for (; sp < nsplit; ++sp) {
                const float2 u = pr[sp * st], v = pi[sp * st];
                ae.x = __fadd_rn(ae.x, u.x);
                ae.y = __fadd_rn(ae.y, u.y);
                db.x = __fadd_rn(db.x, v.x);
                db.y = __fadd_rn(db.y, v.y);
            }
            // X[+c] = (a - b) + j (d + e), X[-c] = (a + b) + j (d - e)
            const float2 Xp = make_float2(__fsub_rn(ae.x, db.y), __fadd_rn(db.x, ae.y));
            const float2 Xm = make_float2(__fadd_rn(ae.x, db.y), __fsub_rn(db.x, ae.y));
            if (wp) {
                if constexpr (ABS) oa[kp] = cabs_rn(Xp);
                else o[kp] = Xp;
            }
            if (wm) {
                if constexpr (ABS) oa[km] = cabs_rn(Xm);
                else o[km] = Xm;
            }
        }
    }
    // bin 0 (if in the window): the DC tiles in a fixed order, warp 0 of the y = 0 block
    int64_t k0 = (-(int64_t)p0) % N;
    if (k0 < 0) k0 += N;
    if (threadIdx.x < 32 && k0 < nbins && blockIdx.y == 0) {
        float sr = 0.f, si = 0.f;
        for (int g = threadIdx.x; g < gy; g += 32) {
            const float2 v = dc[(int64_t)g * ncols + col];
            sr = __fadd_rn(sr, v.x);
            si = __fadd_rn(si, v.y);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sr = __fadd_rn(sr, __shfl_xor_sync(0xffffffffu, sr, off));
            si = __fadd_rn(si, __shfl_xor_sync(0xffffffffu, si, off));
        }
        if (threadIdx.x == 0) {
            if constexpr (ABS) oa[k0] = cabs_rn(make_float2(sr, si));
            else o[k0] = make_float2(sr, si);
        }
    }
}

// Paired adjoint B operand: with W^(-c i) = conj(W^(c i)) the bins +c and -c
// of dA enter G_l[i] = sum_p conj(S[p][i]) dA[l][p] as
//     conj(S) x + S y = S_r u_r + S_i v_i + j (S_r u_i - S_i v_r),
// x = dA[l][+c], y = dA[l][-c] (0 where the bin is not in the window, y = 0
// when -c = +c), u = x + y, v = x - y.  Row (kb, 2 l) holds frequencies
// 16 kb .. 16 kb + 15 as [u_r hi, lo, v_i hi, lo] and row (kb, 2 l + 1) as
// [u_i hi, lo, -v_r hi, lo] (bf16), against the A rows' [S_r, S_r, S_i, S_i].
// One thread per (lag, frequency), coalesced over the frequencies.
__global__ void __launch_bounds__(256) k_pack_adjoint_pair(const float2 *__restrict__ dA, int N, int p0, int nbins,
                                                            int nlags, int slots, int kblocks, uint2 *__restrict__ B) {
    const int64_t total = (int64_t)nlags * kblocks * 16;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = e / ((int64_t)kblocks * 16);
        const int c = (int)(e - l * kblocks * 16);  // frequency
        float2 x = make_float2(0.f, 0.f), y = x;
        if (c < slots) {
            int64_t kx = ((int64_t)c - p0) % N;
            if (kx < 0) kx += N;
            int64_t ky = (-(int64_t)c - p0) % N;
            if (ky < 0) ky += N;
            const bool self_conj = (2LL * c) % N == 0;  // -c = +c (mod N)
            if (kx < nbins) x = dA[l * nbins + kx];
            if (!self_conj && ky < nbins) y = dA[l * nbins + ky];
        }
        const float ur = x.x + y.x, ui = x.y + y.y, vr = x.x - y.x, vi = x.y - y.y;
        uint32_t h0, l0, h1, l1;
        split2(ur, vi, h0, l0);   // [u_r hi, v_i hi], [u_r lo, v_i lo]
        split2(ui, -vr, h1, l1);  // [u_i hi, -v_r hi], [u_i lo, -v_r lo]
        const int kb = c >> 4, k = c & 15;
        // K order per frequency: [hi(u), lo(u), hi(v), lo(v)]
        B[((int64_t)kb * 2 * nlags + 2 * l) * 16 + k] =
            make_uint2(__byte_perm(h0, l0, 0x5410), __byte_perm(h0, l0, 0x7632));
        B[((int64_t)kb * 2 * nlags + 2 * l + 1) * 16 + k] =
            make_uint2(__byte_perm(h1, l1, 0x5410), __byte_perm(h1, l1, 0x7632));
    }
}

// Two-level angle table: entry j < nth is (cos, sin)((pi/2) 256 j / N), entry
// nth + j (j < 256) is (cos, sin)((pi/2) j / N); fp64, rounded to fp32.
__global__ void k_angles(int N, int nth, float2 *__restrict__ ang) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nth + R_LO) return;
    const int64_t r = e < nth ? (int64_t)e * R_LO : (int64_t)(e - nth);
    const double a = 1.5707963267948966 * ((double)r / (double)N);
    ang[e] = (r == 0) ? make_float2(1.f, 0.f) : make_float2(__double2float_rn(cos(a)), __double2float_rn(sin(a)));
}

// The paired contraction's A operand for a whole plan: row (kb, m) holds the
// 64 K entries of row m (slot s = m / 2, frequency c = p0 + s; m even the R
// row, odd the I row) for samples 16 kb .. 16 kb + 15, in the chunk order of
// gen_conj_chunk, with each twiddle from the two-level table (no rotation)
// and its signs from the exact twiddle index.  Rows past 2 S are zero.
__global__ void k_atab(int N, int p0, int S, int rows, int kblocks, const float2 *__restrict__ ang, int nth,
                       uint4 *__restrict__ out) {
    const int64_t total = (int64_t)kblocks * (rows / 2) * 8;  // (kb, slot, chunk)
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e & 7);
        const int64_t r = e >> 3;
        const int sl = (int)(r % (rows / 2));
        const int64_t kb = r / (rows / 2);
        uint4 re = make_uint4(0u, 0u, 0u, 0u), im = re;
        if (sl < S) {
            int64_t c = ((int64_t)p0 + sl) % N;
            if (c < 0) c += N;
            const int64_t i0 = (kb * 16 + 2 * t) % N, i1 = (i0 + 1) % N;
            const uint32_t ua = 4u * (uint32_t)((c * i0) % N), ub = 4u * (uint32_t)((c * i1) % N);
            const float2 wa = tw_table_g(ua, (uint32_t)N, ang, nth), wb = tw_table_g(ub, (uint32_t)N, ang, nth);
            gen_conj_chunk((float)ua, (float)ub, wa, wb, (float)N, re, im);
        }
        out[(kb * rows + 2 * sl) * 8 + t] = re;
        out[(kb * rows + 2 * sl + 1) * 8 + t] = im;
    }
}

// The paired adjoint's A rows as a table: [K block][row] of 128-byte rows,
// row i (a sample; rows past N repeat i mod N) holding for frequencies c =
// 16 kb + 2 t and c + 1 the sign words [S_r, S_r], [S_i, S_i] of
// S = sigma(W^(c i)) (the integer quadrant rule), exactly what the adjoint's
// producer warps write.
__global__ void k_atab_adj(int N, int rows, int kblocks, uint4 *__restrict__ out) {
    const int64_t total = (int64_t)kblocks * rows * 8;  // (kb, row, chunk)
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e & 7);
        const int64_t r = e >> 3;
        const int64_t row = r % rows, kb = r / rows;
        const int64_t i = row % N;
        const int64_t c0 = (kb * 16 + 2 * t) % N, c1 = c0 + 1 == N ? 0 : c0 + 1;
        uint32_t sra, sia, srb, sib;
        sign_bits(4u * (uint32_t)((c0 * i) % N), (uint32_t)N, sra, sia);
        sign_bits(4u * (uint32_t)((c1 * i) % N), (uint32_t)N, srb, sib);
        out[r * 8 + t] = make_uint4(sra, sia, srb, sib);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

cudaError_t make_tmap(void *base, int64_t rows, CUtensorMap *map, int box_rows = TN) {
    auto enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {64, (cuuint64_t)rows};
    cuuint64_t strides[1] = {128};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Output (or split partials) as a 3-D fp32 tensor {2 nbins rows, ncols, nsplit},
// box 32 rows x 16 columns x 1 split, no swizzle: the epilogue warps' bulk
// stores / adds (one warp's 32 TMEM lanes, a 16-column group).  Needs 2 nbins * 4 bytes to be a multiple of 16 (nbins even).
cudaError_t make_out_map(void *base, int nbins, int ncols, int nsplit, CUtensorMap *map, int box_cols = 16) {
    auto enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t rows = 2ull * nbins;
    cuuint64_t dims[3] = {rows, (cuuint64_t)ncols, (cuuint64_t)nsplit};
    cuuint64_t strides[2] = {rows * 4, rows * 4 * (cuuint64_t)ncols};
    cuuint32_t box[3] = {32, (cuuint32_t)box_cols, 1};  // one epilogue warp's 32 rows x 16 (paired: 32) columns
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The same for an output of `rows` fp32 rows per column (the paired adjoint's
// G: one row per sample), box 32 rows x 32 columns.  Needs rows * 4 bytes to
// be a multiple of 16.
cudaError_t make_out_rows_map(void *base, int64_t rows, int ncols, int nsplit, CUtensorMap *map) {
    auto enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    cuuint64_t dims[3] = {(cuuint64_t)rows, (cuuint64_t)ncols, (cuuint64_t)nsplit};
    cuuint64_t strides[2] = {(cuuint64_t)rows * 4, (cuuint64_t)rows * 4 * (cuuint64_t)ncols};
    cuuint32_t box[3] = {32, 32, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int nth_for(int N) { return (N - 1) / R_LO + 1; }

int max_cols(const ndft_desc &d) { return (int)std::max<int64_t>(d.max_lags, d.max_batch); }

// Splits along the sample axis: none when the tiles alone fill two waves;
// otherwise the split count in [2 waves, capacity] with the best wave
// quantisation (smallest on ties).  `cap_units` bounds split * tiles by the
// partials buffer.
int choose_split(int64_t tiles, int kblocks, int sm, int tune, int64_t cap_units) {
    const int cap = (int)std::max<int64_t>(1, std::min<int64_t>(kMaxSplit, cap_units / tiles));
    int s;
    if (tune > 0) {
        s = std::min(tune, cap);
    } else if (tiles >= 2LL * sm) {
        s = 1;
    } else {
        const int lo = (int)std::min<int64_t>((2LL * sm + tiles - 1) / tiles, cap);
        s = lo;
        double best = 0.0;
        for (int c = lo; c <= cap; ++c) {
            const int64_t units = tiles * c;
            const double eff = (double)units / (double)(((units + sm - 1) / sm) * sm);
            if (eff > best + 1e-9) {
                best = eff;
                s = c;
            }
        }
    }
    return std::max(1, std::min(s, std::max(1, kblocks / 4)));
}

// max_blocks > 0 bounds the single-problem grid to about that many blocks (its
// y extent shrinks and the blocks loop over the K-block tiles).
cudaError_t launch_pack(const PackProb *probs, const int64_t *prefix, int nprob, const PackProb &single,
                        int64_t rows, uint32_t flags, bool caf, const void *a_base, const void *r_base, void *B, int sm,
                        cudaStream_t s, int32_t *err, int max_blocks = 0) {
    const int threads = 256;
    if (!probs) {
        const int gx = (single.ncols + 31) / 32;
        const int gy = (single.kblocks + kPackKb - 1) / kPackKb;
        int grid_y = std::min(gy, 65535);
        if (max_blocks > 0) grid_y = std::max(1, std::min(grid_y, max_blocks / gx));
        k_pack_single<<<dim3(gx, grid_y), threads, 0, s>>>(single, flags, caf, static_cast<const float2 *>(a_base),
                                                           static_cast<const float2 *>(r_base),
                                                           static_cast<uint4 *>(B), gy, err);
        return cudaGetLastError();
    }
    const int64_t want = (rows * 8 + threads - 1) / threads;
    const int blocks = (int)std::min<int64_t>(want, (int64_t)sm * 32);
    k_pack<<<std::max(blocks, 1), threads, 0, s>>>(probs, prefix, nprob, single, rows, flags, caf,
                                                   static_cast<const float2 *>(a_base),
                                                   static_cast<const float2 *>(r_base), static_cast<uint4 *>(B), err);
    return cudaGetLastError();
}

template <int MH, bool BT = false, int ADJ = 0, bool PAIR = false, bool ATAB = false>
cudaError_t launch_gemm(const Plan &p, const Problem &single, const Problem *probs, const Unit *units,
                        int64_t nunits, float *out_base, const CUtensorMap *omap, cudaStream_t s,
                        const void *amap = nullptr, const void *bmap = nullptr) {
    constexpr size_t smem = TileOf<PAIR, MH>::type::kSmemTotal;
    auto kern = k_ternary_gemm<MH, BT, ADJ, PAIR, ATAB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const CUtensorMap *map = static_cast<const CUtensorMap *>(bmap ? bmap : p.tmap_host);
    const int chunk = p.tune_chunk > 0 ? p.tune_chunk : (PAIR ? kChunkPair : kChunk);
    CUtensorMap none;
    std::memset(&none, 0, sizeof(none));
    const CUtensorMap &om = omap ? *omap : none;
    const int out_tma = omap ? 1 : 0;
    timer_begin(p, s);
    const int grid = (int)std::min<int64_t>(nunits, p.sm_count);
    if (ATAB && !amap) amap = p.tmap_a;  // the forward table unless another is given
    if (ATAB && !amap) return cudaErrorInvalidValue;
    const CUtensorMap &am = ATAB ? *static_cast<const CUtensorMap *>(amap) : none;
    kern<<<grid, gemm_threads(PAIR, ATAB), smem, s>>>(*map, om, out_tma, single, probs, units, nunits, chunk,
                                                      p.test_starve, out_base, p.err, am);
    e = cudaGetLastError();
    timer_end(p, s);
    return e;
}

// The 2-SM pair tile: one unit per pair, 2 x min(units, SMs / 2) CTAs in clusters of 2.
template <bool ATAB = false, int BM = kBTma>
cudaError_t launch_gemm_pair(const Plan &p, const Problem &single, int64_t nunits, float *out_base,
                             const CUtensorMap *omap, cudaStream_t s, const BGen *bgen = nullptr) {
    constexpr size_t smem = pair2::kSmemTotal;
    if (ATAB && !p.tmap_a2) return cudaErrorInvalidValue;
    if (BM != kBTma && !bgen) return cudaErrorInvalidValue;
    BGen bg{};
    if (bgen) bg = *bgen;
    auto kern = k_ternary_gemm_pair<ATAB, BM>;
    constexpr int threads = pair_threads(BM);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const CUtensorMap *map = static_cast<const CUtensorMap *>(p.tmap_host2);  // 128-row box
    const int chunk = p.tune_chunk > 0 ? p.tune_chunk : kChunk;
    CUtensorMap none;
    std::memset(&none, 0, sizeof(none));
    const CUtensorMap &om = omap ? *omap : none;
    const int out_tma = omap ? 1 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * std::min<int64_t>(nunits, p.sm_count / 2)));
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    timer_begin(p, s);
    const CUtensorMap &am = (ATAB && p.tmap_a2) ? *static_cast<const CUtensorMap *>(p.tmap_a2) : none;
    e = cudaLaunchKernelEx(&cfg, kern, *map, om, out_tma, single, nunits, chunk, p.test_starve, out_base, p.err, am,
                           bg);
    timer_end(p, s);
    return e;
}

// Tile shape (tuning key 1): 256 rows in one CTA (one accumulator pair), 128
// rows with two accumulators used in turn (128), or the 256 x 256 tile on a
// 2-SM pair (258, cta_group::2).  The default (0) is the 2-SM pair for the
// conjugate-paired contraction with its A operand from the plan's table and the
// one-CTA 256-row tile everywhere else.
int tile_halves(const Plan &p) { return p.tune_cols == 128 ? 1 : 2; }
bool tile_pair(const Plan &p) { return p.tune_cols == 258; }

struct TernLayout {
    int kblocks;
    int64_t b_rows;
    size_t b_bytes;
    size_t part_bytes;
    size_t dc_bytes;  // paired form: bin-0 sums per packing tile (or item row) and column, then item flags
    size_t dc_flag_off;
};

int pair_kblocks(int N) { return (N + 15) / 16; }
int pair_pack_tiles(int N) { return (pair_kblocks(N) + kPairPackKb - 1) / kPairPackKb; }

// Frequencies 1 .. S that the bin window p0 .. p0 + nbins - 1 (mod N) folds
// onto, c(p) = min(p, N - p); S = max c over the window.
int pair_slots_for(int N, int p0, int nbins) {
    int64_t cmax = 0;
    for (int k = 0; k < nbins; ++k) {
        int64_t p = ((int64_t)p0 + k) % N;
        if (p < 0) p += N;
        cmax = std::max<int64_t>(cmax, std::min<int64_t>(p, N - p));
    }
    return (int)cmax;
}

TernLayout layout_for(const ndft_desc &d, int sm) {
    TernLayout L;
    L.kblocks = (d.n + 7) / 8;
    const int cols = max_cols(d);
    // the unpaired layout (8 samples x 8 entries per row, one row per column)
    // or the paired one (16 samples x 4 entries, two rows per column)
    L.b_rows = std::max<int64_t>((int64_t)L.kblocks * cols, (int64_t)pair_kblocks(d.n) * 2 * cols);
    L.b_bytes = (size_t)L.b_rows * 128;
    L.part_bytes = (size_t)4 * sm * 256 * TN * sizeof(float);  // 4 waves of 256 x 256 partial tiles
    // bin-0 partial rows: one per packing tile, or (B packed inside the pair
    // tile) one per split and block of 16 K blocks, at most tiles + 34 with
    // at most kMaxSplit splits; then the flags of that mode's work items
    // (rows x column blocks of 64, at most cols / 64 + 2 of them)
    const int64_t dc_rows = pair_pack_tiles(d.n) + kMaxSplit + 8;
    L.dc_flag_off = ((size_t)dc_rows * cols * sizeof(float2) + 255) / 256 * 256;
    L.dc_bytes = L.dc_flag_off + ((size_t)(1 + dc_rows * (cols / 64 + 2)) * sizeof(int32_t) + 255) / 256 * 256;
    // the paired contraction writes at least one split of partials [2 cols][2 S]
    // (the fold writes the output): room for it at the plan's largest call
    const int S = pair_slots_for(d.n, d.p0, d.nbins ? d.nbins : d.n);
    if (S > 0) L.part_bytes = std::max(L.part_bytes, (size_t)2 * cols * 2 * S * sizeof(float));
    return L;
}



// Device-side description of a batched plan (one allocation, laid out by
// ternary_batched_init): Problem[ncpi], PackProb[ncpi], int64 prefix[ncpi + 1]
// (first packed row), int64 tile prefix[ncpi + 1] (first pack tile),
// Unit[nunits].
struct BatchedLayout {
    size_t probs, packs, prefix, tprefix, units, total;
};

BatchedLayout batched_layout(int ncpi, int64_t nunits) {
    BatchedLayout b;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    b.probs = 0;
    b.packs = al(b.probs + (size_t)ncpi * sizeof(Problem));
    b.prefix = al(b.packs + (size_t)ncpi * sizeof(PackProb));
    b.tprefix = al(b.prefix + (size_t)(ncpi + 1) * sizeof(int64_t));
    b.units = al(b.tprefix + (size_t)(ncpi + 1) * sizeof(int64_t));
    b.total = al(b.units + (size_t)nunits * sizeof(Unit));
    return b;
}

}  // namespace

bool ternary_supported(const ndft_desc &d) {
    return d.form == NDFT_FORM_TERNARY_GEMM && d.prec == NDFT_PREC_BF16X2 && d.n >= 1 && d.n <= kMaxN;
}

size_t ternary_ws_bytes(const ndft_desc &d, int sm) {
    if (!ternary_supported(d)) return 0;
    const TernLayout L = layout_for(d, sm);
    return L.b_bytes + L.part_bytes + L.dc_bytes;
}

cudaError_t ternary_plan_init(Plan &p, cudaStream_t s) {
    if (!ternary_supported(p.d)) return cudaErrorNotSupported;
    const int N = p.d.n;
    const int nth = nth_for(N);
    cudaError_t e;
    if ((e = cudaMalloc(&p.ang, (size_t)(nth + R_LO) * sizeof(float2))) != cudaSuccess) return e;
    p.table_bytes += (size_t)(nth + R_LO) * sizeof(float2);
    k_angles<<<(nth + R_LO + 255) / 256, 256, 0, s>>>(N, nth, p.ang);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const TernLayout L = layout_for(p.d, p.sm_count);
    p.b_bytes = L.b_bytes;
    p.part_bytes = L.part_bytes;
    p.dc_bytes = L.dc_bytes;
    p.dc_flag_off = L.dc_flag_off;
    p.pair_slots = pair_slots_for(N, p.d.p0, p.d.nbins);
    // the paired A operand as a table when it is modest (it depends on the
    // window and N only; the contraction then needs no producer warps)
    if (p.pair_slots > 0) {
        const int rows = (2 * p.pair_slots + 255) / 256 * 256;
        const int kbp = pair_kblocks(N);
        const size_t bytes = (size_t)kbp * rows * 128;
        if (bytes <= kAtabMaxBytes && (int64_t)kbp * rows < (1LL << 31)) {
            if ((e = cudaMalloc(&p.atab, bytes)) != cudaSuccess) return e;
            p.atab_bytes = bytes;
            p.atab_ld = rows;
            p.table_bytes += bytes;
            const int64_t items = (int64_t)kbp * (rows / 2) * 8;
            const int blocks = (int)std::min<int64_t>((items + 255) / 256, (int64_t)p.sm_count * 32);
            k_atab<<<blocks, 256, 0, s>>>(N, 1, p.pair_slots, rows, kbp, p.ang, nth, static_cast<uint4 *>(p.atab));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            p.tmap_a = std::aligned_alloc(64, sizeof(CUtensorMap));
            if (!p.tmap_a) return cudaErrorMemoryAllocation;
            if ((e = make_tmap(p.atab, (int64_t)kbp * rows, static_cast<CUtensorMap *>(p.tmap_a))) != cudaSuccess)
                return e;
            p.tmap_a2 = std::aligned_alloc(64, sizeof(CUtensorMap));  // 128-row box for the 2-SM pair tile
            if (!p.tmap_a2) return cudaErrorMemoryAllocation;
            if ((e = make_tmap(p.atab, (int64_t)kbp * rows, static_cast<CUtensorMap *>(p.tmap_a2), TN / 2)) !=
                cudaSuccess)
                return e;
        }
        // CAF plans: the paired adjoint's sign rows as a table too ([frequency
        // block][sample row], 277 MB for 65536 samples and 513 frequencies)
        const int kba = (p.pair_slots + 1 + 15) / 16;
        const int arows = (N + 255) / 256 * 256;
        const size_t abytes = (size_t)kba * arows * 128;
        if (p.d.max_lags > 0 && abytes <= kAtabMaxBytes && (int64_t)kba * arows < (1LL << 31)) {
            if ((e = cudaMalloc(&p.atab_adj, abytes)) != cudaSuccess) return e;
            p.atab_adj_bytes = abytes;
            p.atab_adj_ld = arows;
            p.table_bytes += abytes;
            const int64_t items = (int64_t)kba * arows * 8;
            const int blocks = (int)std::min<int64_t>((items + 255) / 256, (int64_t)p.sm_count * 32);
            k_atab_adj<<<blocks, 256, 0, s>>>(N, arows, kba, static_cast<uint4 *>(p.atab_adj));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            p.tmap_adj = std::aligned_alloc(64, sizeof(CUtensorMap));
            if (!p.tmap_adj) return cudaErrorMemoryAllocation;
            if ((e = make_tmap(p.atab_adj, (int64_t)kba * arows, static_cast<CUtensorMap *>(p.tmap_adj))) !=
                cudaSuccess)
                return e;
        }
    }
    p.tmap_host = std::aligned_alloc(64, sizeof(CUtensorMap));  // CUtensorMap wants 64-byte alignment
    if (!p.tmap_host) return cudaErrorMemoryAllocation;
    if ((e = make_tmap(p.ws, std::max<int64_t>(L.b_rows, 1), static_cast<CUtensorMap *>(p.tmap_host))) !=
        cudaSuccess)
        return e;
    p.tmap_host2 = std::aligned_alloc(64, sizeof(CUtensorMap));  // 128-row box for the pair tile
    if (!p.tmap_host2) return cudaErrorMemoryAllocation;
    if ((e = make_tmap(p.ws, std::max<int64_t>(L.b_rows, 1), static_cast<CUtensorMap *>(p.tmap_host2), TN / 2)) !=
        cudaSuccess)
        return e;
    // side stream and fork / join events of the two-part contraction; the packing
    // kernel asks for the largest shared-memory carveout, so that an SM running
    // its blocks is configured to take a contraction CTA beside them
    if ((e = cudaFuncSetAttribute(k_pack_single, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
        return e;
    if ((e = cudaStreamCreateWithFlags(&p.side, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&p.ev_fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    return cudaEventCreateWithFlags(&p.ev_join, cudaEventDisableTiming);
}

// Packs columns [c0, c0 + nc) of a single problem into the B rows from b_row0
// on (laid out as a problem of nc columns).
static cudaError_t pack_cols(Plan &p, PackProb pp, bool caf, int c0, int nc, int64_t b_row0, const void *a_base,
                             const void *r_base, cudaStream_t s, int max_blocks) {
    if (caf) pp.lag0 += c0;  // the lag window fits in int32 (checked at the boundary)
    else pp.a_off += (int64_t)c0 * pp.ldx;
    pp.ncols = nc;
    pp.row0 = b_row0;
    return launch_pack(nullptr, nullptr, 0, pp, (int64_t)pp.kblocks * nc, p.d.flags, caf, a_base, r_base, p.ws,
                       p.sm_count, s, p.err, max_blocks);
}

// Contraction of nc packed columns (B rows from b_row0 on) into out
// ([nc][nbins] complex), with the ordered split-K sum when the sample axis is
// split.
static cudaError_t gemm_cols(Plan &p, int nc, int64_t b_row0, void *out, cudaStream_t s, int *launches) {
    const int N = p.d.n, nb = p.d.nbins;
    const TernLayout L = layout_for(p.d, p.sm_count);
    Problem P{};
    P.N = N;
    P.p0 = p.d.p0;
    P.nbins = nb;
    P.ncols = nc;
    P.kblocks = L.kblocks;
    const bool pair = tile_pair(p);
    const int MH = tile_halves(p);
    const int rows = 128 * MH;
    P.mtiles = (2 * nb + rows - 1) / rows;
    P.ntiles = (nc + TN - 1) / TN;
    // scheduled units per split and the slots that run them (a 2-SM pair per unit
    // with the pair tile)
    const int64_t tiles = (int64_t)P.mtiles * P.ntiles;
    const int slots = pair ? p.sm_count / 2 : p.sm_count;
    const int64_t cap_units = (int64_t)(L.part_bytes / ((size_t)rows * TN * sizeof(float)));
    P.nsplit = choose_split(tiles, L.kblocks, slots, p.tune_split, cap_units);
    P.b_row0 = b_row0;
    P.ld = 2LL * nb;
    P.split_stride = (int64_t)nc * 2 * nb;
    P.ang = p.ang;
    P.nth = nth_for(N);
    P.out_off = 0;
    float *part = reinterpret_cast<float *>(static_cast<unsigned char *>(p.ws) + L.b_bytes);
    const bool abs_out = (p.d.flags & NDFT_F_ABS_OUT) != 0;  // |A| is formed by the split sum
    float *out_base = (P.nsplit == 1 && !abs_out) ? static_cast<float *>(out) : part;
    const int64_t nunits = tiles * P.nsplit;
    // bulk tensor stores / adds for the epilogue when the rows are 16-byte multiples
    alignas(64) CUtensorMap omap;
    const bool tma_out = (nb % 2 == 0) && p.tune_drain == 0 &&
                         make_out_map(out_base, nb, nc, P.nsplit, &omap) == cudaSuccess;
    const CUtensorMap *om = tma_out ? &omap : nullptr;
    cudaError_t e;
    if (pair) e = launch_gemm_pair(p, P, nunits, out_base, om, s);
    else if (MH == 2) e = launch_gemm<2>(p, P, nullptr, nullptr, nunits, out_base, om, s);
    else e = launch_gemm<1>(p, P, nullptr, nullptr, nunits, out_base, om, s);
    if (e != cudaSuccess) return e;
    *launches += 1;
    p.last_variant = 1;
    p.last_nsplit = P.nsplit;
    p.last_tile = pair ? 258 : rows;
    if (abs_out) {
        *launches += 1;
        return launch_reduce_abs(reinterpret_cast<const float2 *>(part), P.nsplit, (int64_t)nc * nb,
                                 static_cast<float *>(out), s);
    }
    if (P.nsplit > 1) {
        *launches += 1;
        return launch_reduce_splits(part, P.nsplit, (int64_t)nc * 2 * nb, static_cast<float *>(out), s);
    }
    return cudaSuccess;
}

// Columns of the first part when a problem runs in two column parts: the
// tuning value (a multiple of TN), 1 for one part, or by default half the
// columns rounded down to TN once there are at least 2 TN.
static int first_part_cols(const Plan &p, int ncols) {
    if (!p.side || p.tune_parts == 1 || (p.d.flags & NDFT_F_ABS_OUT)) return 0;
    const int h0 = p.tune_parts > 1 ? p.tune_parts : std::max(TN, (ncols / 2) / TN * TN);
    return (ncols >= 2 * TN && h0 < ncols) ? h0 : 0;
}

// Grid of the second part's packing: two blocks of 256 threads per SM, which
// fit beside one contraction CTA (448 threads, under 48 K registers, the shared
// memory untouched), so the packing runs under the first part's contraction.
constexpr int kPackBlocksPerSm = 2;

// Conjugate-paired contraction of ncols columns: rows = the R / I rows of
// frequencies 1 .. S, columns = (col, r/i), K = 16 samples per block; the
// split partials always go to the workspace, and the fold writes the output
// (bin 0 from the packing kernel's DC sums).
static cudaError_t pair_cols(Plan &p, const PackProb &pp0, bool caf, int ncols, const void *a_base,
                             const void *r_base, void *out, cudaStream_t s, int *launches) {
    const int N = p.d.n, S = p.pair_slots;
    const int kblocks = pair_kblocks(N);
    const int gy = pair_pack_tiles(N);
    float *part = reinterpret_cast<float *>(static_cast<unsigned char *>(p.ws) + p.b_bytes);
    float2 *dc = reinterpret_cast<float2 *>(static_cast<unsigned char *>(p.ws) + p.b_bytes + p.part_bytes);
    PackProb pp = pp0;
    pp.kblocks = kblocks;
    pp.ncols = ncols;
    pp.row0 = 0;
    const int64_t tiles = (int64_t)((2 * S + 255) / 256) * ((2LL * ncols + TN - 1) / TN);
    const int64_t cap_units = (int64_t)(p.part_bytes / ((size_t)256 * TN * sizeof(float)));
    // A from the plan's table: the 2-SM pair tile unless key 1 asks for the one-CTA tile
    const bool atab = p.atab && p.tune_atab == 0;
    const bool pair_tile = atab && (p.tune_cols == 0 || tile_pair(p));
    const int nsplit = choose_split(tiles, kblocks, pair_tile ? p.sm_count / 2 : p.sm_count, p.tune_split, cap_units);
    // B formed inside the pair tile (key 8 = 2), its bin-0 sums one row per split
    const bool bgen =
        pair_tile && p.tune_bgen == 2 && (size_t)nsplit * ncols * sizeof(float2) <= p.dc_flag_off;
    // B packed just in time by the pair tile's own warps (key 8 = 3, and the
    // default on the pair tile): items of 16 K blocks x 64 columns, bin-0 sums
    // one row per split and block
    const int jmax = ((kblocks + nsplit - 1) / nsplit + 15) / 16;
    const int ncx = 2 * ((ncols + 127) / 128);
    const int64_t nitems = (int64_t)nsplit * jmax * ncx;
    int32_t *flags = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(dc) + p.dc_flag_off);
    const bool ahead = pair_tile && (p.tune_bgen == 3 || p.tune_bgen == 0) &&
                       (size_t)nsplit * jmax * ncols * sizeof(float2) <= p.dc_flag_off &&
                       (size_t)(1 + nitems) * sizeof(int32_t) <= p.dc_bytes - p.dc_flag_off;
    if (ahead) {
        cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)(1 + nitems) * sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
    } else if (!bgen) {
        const int gx = (ncols + 31) / 32;
        k_pack_pair<<<dim3(gx, std::min(gy, 65535)), 256, 0, s>>>(
            pp, p.d.flags, caf, static_cast<const float2 *>(a_base), static_cast<const float2 *>(r_base),
            static_cast<uint4 *>(p.ws), dc, gy, p.err);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        *launches += 1;
    }
    Problem P{};
    P.N = N;
    P.p0 = 1;
    P.nbins = S;
    P.ncols = 2 * ncols;
    P.kblocks = kblocks;
    P.mtiles = (2 * S + 255) / 256;
    P.ntiles = (P.ncols + TN - 1) / TN;
    P.nsplit = nsplit;
    P.b_row0 = 0;
    P.ld = 2LL * S;
    P.split_stride = (int64_t)P.ncols * 2 * S;
    P.ang = p.ang;
    P.nth = nth_for(N);
    P.out_off = 0;
    alignas(64) CUtensorMap omap;
    const bool tma_out =
        (S % 2 == 0) && p.tune_drain == 0 && make_out_map(part, S, P.ncols, P.nsplit, &omap, 32) == cudaSuccess;
    P.a_ld = p.atab_ld;
    cudaError_t e;
    if (pair_tile) {
        // the 2-SM pair tile: two accumulators in turn, the fold-out under the next chain
        alignas(64) CUtensorMap omap16;
        const bool tma16 =
            (S % 2 == 0) && p.tune_drain == 0 && make_out_map(part, S, P.ncols, P.nsplit, &omap16) == cudaSuccess;
        if (bgen || ahead) {
            BGen bg{pp, static_cast<const float2 *>(a_base), static_cast<const float2 *>(r_base), dc,
                    p.d.flags, caf ? 1 : 0};
            if (ahead) {
                bg.B = static_cast<uint4 *>(p.ws);
                bg.ctr = flags;
                bg.nitems = nitems;
                bg.jmax = jmax;
                bg.ncx = ncx;
                bg.look = p.tune_look > 0 ? p.tune_look : 4;
                e = launch_gemm_pair<true, kBAhead>(p, P, tiles * P.nsplit, part, tma16 ? &omap16 : nullptr, s, &bg);
            } else {
                e = launch_gemm_pair<true, kBForm>(p, P, tiles * P.nsplit, part, tma16 ? &omap16 : nullptr, s, &bg);
            }
        } else {
            e = launch_gemm_pair<true>(p, P, tiles * P.nsplit, part, tma16 ? &omap16 : nullptr, s);
        }
    } else if (atab) {
        e = launch_gemm<2, false, 0, true, true>(p, P, nullptr, nullptr, tiles * P.nsplit, part,
                                                 tma_out ? &omap : nullptr, s);
    } else {
        e = launch_gemm<2, false, 0, true>(p, P, nullptr, nullptr, tiles * P.nsplit, part, tma_out ? &omap : nullptr,
                                           s);
    }
    if (e != cudaSuccess) return e;
    *launches += 1;
    p.last_variant = 2;
    p.last_nsplit = P.nsplit;
    p.last_tile = pair_tile ? 258 : 256;
    const dim3 fgrid(ncols, (S + kFoldBins - 1) / kFoldBins);
    // bin-0 partials: per split and block, per split, or per packing tile
    const int dc_rows = ahead ? P.nsplit * jmax : bgen ? P.nsplit : gy;
    if (p.d.flags & NDFT_F_ABS_OUT)
        k_pair_fold<true><<<fgrid, kFoldBins, 0, s>>>(part, P.nsplit, P.split_stride, S, N, p.d.p0, p.d.nbins, dc,
                                                      dc_rows, ncols, out, p.err);
    else
        k_pair_fold<false><<<fgrid, kFoldBins, 0, s>>>(part, P.nsplit, P.split_stride, S, N, p.d.p0, p.d.nbins, dc,
                                                       dc_rows, ncols, out, p.err);
    *launches += 1;
    return cudaGetLastError();
}

// Whether a call of ncols columns runs conjugate-paired: the plan's window
// folds onto frequencies 1 .. S, the default tile and one part are in use,
// the partials of one split fit, and the paired contraction issues fewer
// K-block steps than the unpaired one.
static bool use_pair(const Plan &p, int ncols) {
    if (p.tune_pair == 1 || p.pair_slots < 1 || tile_halves(p) != 2 || first_part_cols(p, ncols)) return false;
    if (tile_pair(p) && !(p.atab && p.tune_atab == 0)) return false;  // the pair tile needs the A table
    const int64_t S = p.pair_slots, nb = p.d.nbins, N = p.d.n;
    if ((size_t)2 * ncols * 2 * S * sizeof(float) > p.part_bytes) return false;
    if ((size_t)pair_pack_tiles((int)N) * ncols * sizeof(float2) > p.dc_flag_off) return false;
    if (p.tune_pair == 2) return true;
    const int64_t paired = ((2 * S + 255) / 256) * ((2LL * ncols + TN - 1) / TN) * (int64_t)pair_kblocks((int)N);
    const int64_t plain = ((2 * nb + 255) / 256) * (((int64_t)ncols + TN - 1) / TN) * ((N + 7) / 8);
    return paired < plain;
}

static cudaError_t run_single(Plan &p, const PackProb &pp, bool caf, int ncols, const void *a_base,
                              const void *r_base, void *out, cudaStream_t s, int *launches) {
    if (use_pair(p, ncols)) return pair_cols(p, pp, caf, ncols, a_base, r_base, out, s, launches);
    const int h0 = first_part_cols(p, ncols);
    cudaError_t e;
    if (h0 == 0) {
        if ((e = pack_cols(p, pp, caf, 0, ncols, 0, a_base, r_base, s, 0)) != cudaSuccess) return e;
        *launches += 1;
        return gemm_cols(p, ncols, 0, out, s, launches);
    }
    // Two column parts.  Part 0 is packed on s; part 1 is packed on the plan's
    // side stream once part 0's packing is done (and with it everything before
    // on s, such as the last call's contraction reading B), during part 0's
    // contraction; part 1's contraction waits for it.  B rows: part 0 first.
    const int h1 = ncols - h0;
    const int64_t row1 = (int64_t)pp.kblocks * h0;
    if ((e = pack_cols(p, pp, caf, 0, h0, 0, a_base, r_base, s, 0)) != cudaSuccess) return e;
    *launches += 1;
    if ((e = cudaEventRecord(p.ev_fork, s)) != cudaSuccess) return e;
    if ((e = gemm_cols(p, h0, 0, out, s, launches)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(p.side, p.ev_fork, 0)) != cudaSuccess) return e;
    if ((e = pack_cols(p, pp, caf, h0, h1, row1, a_base, r_base, p.side, kPackBlocksPerSm * p.sm_count)) !=
        cudaSuccess)
        return e;
    *launches += 1;
    if ((e = cudaEventRecord(p.ev_join, p.side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, p.ev_join, 0)) != cudaSuccess) return e;
    float *out1 = static_cast<float *>(out) + (int64_t)h0 * 2 * p.d.nbins;
    return gemm_cols(p, h1, row1, out1, s, launches);
}

cudaError_t launch_ternary_ndft(Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s, int *launches) {
    PackProb pp{};
    pp.N = p.d.n;
    pp.ncols = (int)batch;
    pp.kblocks = (p.d.n + 7) / 8;
    pp.ldx = p.d.n;
    return run_single(p, pp, false, (int)batch, x, nullptr, X, s, launches);
}

cudaError_t launch_ternary_caf(Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags, void *A,
                               cudaStream_t s, int *launches) {
    PackProb pp{};
    pp.N = p.d.n;
    pp.lag0 = lag0;
    pp.ncols = nlags;
    pp.kblocks = (p.d.n + 7) / 8;
    return run_single(p, pp, true, nlags, s_surv, s_ref, A, s, launches);
}

// Adjoint of the CAF on the tensor cores: G_l[i] = sum_p conj(S[p][i]) dA[l][p]
// as a contraction with rows = (sample, Re/Im), columns = lags and K = bins x
// [dA_hi_r, dA_lo_r, dA_hi_i, dA_lo_i], then ds[i] = sum_l conj(sigma(c_l[i]))
// G_l[i] in the epilogue.  Partials per (lag tile, split) are summed in order.
// Returns cudaErrorNotSupported when the plan's workspace cannot hold it (the
// caller then uses the CUDA-core kernel).
// The paired adjoint contraction: rows = samples, columns = (lag, Re / Im),
// K = frequencies 0 .. S (4 entries each).  Used when the window pairs and
// it issues fewer K-block steps than one row pair per sample over the bins.
// The paired adjoint's A rows from the plan's table (built for CAF plans while
// it stays within kAtabMaxBytes): tuning key 10 = 0 (default) for dL/ds_surv's
// contraction, 2 for both adjoint contractions, 1 for neither.
static bool adj_table(const Plan &p) { return p.atab_adj && p.tmap_adj && p.tune_adj_atab != 1; }

static bool use_pair_adjoint(const Plan &p, int ncols) {
    if (p.tune_pair == 1 || p.pair_slots < 1) return false;
    const int64_t N = p.d.n, nb = p.d.nbins, S1 = p.pair_slots + 1;
    if (p.tune_pair == 2) return true;
    const int64_t paired = ((N + 255) / 256) * ((2LL * ncols + TN - 1) / TN) * ((S1 + 15) / 16);
    const int64_t plain = ((2 * N + 255) / 256) * (((int64_t)ncols + TN - 1) / TN) * ((nb + 15) / 16);
    return paired < plain;
}

// Packs the paired adjoint operand of nc lags of dA into the workspace.
static cudaError_t pack_adjoint_pair(Plan &p, const void *dA, int nc, int kblocks, cudaStream_t s) {
    const int64_t total = (int64_t)nc * kblocks * 16;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)p.sm_count * 16);
    k_pack_adjoint_pair<<<blocks, 256, 0, s>>>(static_cast<const float2 *>(dA), p.d.n, p.d.p0, p.d.nbins, nc,
                                               p.pair_slots + 1, kblocks, static_cast<uint2 *>(p.ws));
    return cudaGetLastError();
}

cudaError_t launch_ternary_adjoint(Plan &p, const void *s_ref, int lag0, int nlags, const void *dA, void *ds,
                                   cudaStream_t s, int *launches) {
    const int N = p.d.n, nb = p.d.nbins;
    if (use_pair_adjoint(p, nlags)) {
        const int kblocks = (p.pair_slots + 1 + 15) / 16;
        Problem P{};
        P.N = N;
        P.p0 = 0;  // frequencies 0, 1, ..
        P.nbins = p.pair_slots + 1;
        P.ncols = 2 * nlags;
        P.kblocks = kblocks;
        P.mtiles = (N + 255) / 256;
        P.ntiles = (P.ncols + TN - 1) / TN;
        const int64_t tiles = (int64_t)P.mtiles * P.ntiles;
        P.nsplit = tiles >= p.sm_count
                       ? 1
                       : (int)std::max<int64_t>(1, std::min<int64_t>(kblocks / 16, (2LL * p.sm_count + tiles - 1) / tiles));
        const int64_t slices = (int64_t)P.ntiles * P.nsplit;
        if ((size_t)kblocks * P.ncols * 128 <= p.b_bytes && (size_t)slices * 2 * N * sizeof(float) <= p.part_bytes) {
            P.b_row0 = 0;
            P.sref = static_cast<const float2 *>(s_ref);
            P.lag0 = lag0;
            P.flags = p.d.flags;
            cudaError_t e = pack_adjoint_pair(p, dA, nlags, kblocks, s);
            if (e != cudaSuccess) return e;
            *launches += 1;
            float *part = reinterpret_cast<float *>(static_cast<unsigned char *>(p.ws) + p.b_bytes);
            if (adj_table(p)) {
                P.a_ld = p.atab_adj_ld;
                e = launch_gemm<2, false, 1, true, true>(p, P, nullptr, nullptr, tiles * P.nsplit, part, nullptr, s,
                                                         p.tmap_adj);
            } else {
                e = launch_gemm<2, false, 1, true>(p, P, nullptr, nullptr, tiles * P.nsplit, part, nullptr, s);
            }
            if (e != cudaSuccess) return e;
            *launches += 2;
            p.last_variant = 2;
            p.last_nsplit = P.nsplit;
            p.last_tile = 256;
            return launch_reduce_splits(part, (int)slices, 2LL * N, static_cast<float *>(ds), s);
        }
    }
    const int kblocks = (nb + 15) / 16;
    const size_t b_need = (size_t)kblocks * nlags * 128;
    Problem P{};
    P.N = N;
    P.p0 = p.d.p0;
    P.nbins = nb;
    P.ncols = nlags;
    P.kblocks = kblocks;
    P.mtiles = (2 * N + 255) / 256;
    P.ntiles = (nlags + TN - 1) / TN;
    const int64_t tiles = (int64_t)P.mtiles * P.ntiles;
    // split the bins only while tiles are scarce, keeping >= 16 K blocks per unit
    // (each unit's epilogue weighs and folds 256 lag columns per row)
    P.nsplit = tiles >= p.sm_count
                   ? 1
                   : (int)std::max<int64_t>(1, std::min<int64_t>(kblocks / 16, (2LL * p.sm_count + tiles - 1) / tiles));
    const int64_t slices = (int64_t)P.ntiles * P.nsplit;
    const size_t part_need = (size_t)slices * 2 * N * sizeof(float);
    if (b_need > p.b_bytes || part_need > p.part_bytes) return cudaErrorNotSupported;
    P.b_row0 = 0;
    P.ld = 0;
    P.split_stride = 0;
    P.out_off = 0;
    P.sref = static_cast<const float2 *>(s_ref);
    P.lag0 = lag0;
    P.flags = p.d.flags;
    const int64_t total = (int64_t)nlags * kblocks * 16;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)p.sm_count * 16);
    k_pack_adjoint<<<blocks, 256, 0, s>>>(static_cast<const float2 *>(dA), nb, nlags, kblocks,
                                          static_cast<uint2 *>(p.ws));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *launches += 1;
    float *part = reinterpret_cast<float *>(static_cast<unsigned char *>(p.ws) + p.b_bytes);
    if ((e = launch_gemm<2, false, 1>(p, P, nullptr, nullptr, tiles * P.nsplit, part, nullptr, s)) !=
        cudaSuccess)
        return e;
    *launches += 2;
    p.last_variant = 1;
    p.last_nsplit = P.nsplit;
    p.last_tile = 256;
    return launch_reduce_splits(part, (int)slices, 2LL * N, static_cast<float *>(ds), s);
}

// The adjoint contraction alone: G_l[i] = sum_p conj(S[p][i]) dA[l][p] for the
// `nc` lags of dA ([nc][nbins] complex), stored as fp32 complex
// [nsplit][nc][N] in the workspace after the packed dA (the forward epilogue
// with rows = (sample, Re/Im) and columns = lags).  The split partials are left
// for the caller, whose fold over lags is linear in G.
namespace {
size_t adjoint_g_offset(int nb, int nc) {
    const size_t b_need = (size_t)((nb + 15) / 16) * nc * 128;
    return (b_need + 1023) & ~(size_t)1023;
}
size_t adjoint_g_need(int N, int nb, int nc, int nsplit) {
    return adjoint_g_offset(nb, nc) + (size_t)nsplit * nc * N * sizeof(float2);
}
}  // namespace

int ternary_adjoint_g_lags(const Plan &p, int nlags) {
    const int N = p.d.n, nb = p.d.nbins;
    int nc = nlags;
    while (nc > 0 && adjoint_g_need(N, nb, nc, 1) > p.ws_alloc) nc = nc > 256 ? (nc - 1) / 256 * 256 : nc / 2;
    return nc;
}

cudaError_t launch_ternary_adjoint_g(Plan &p, int nc, const void *dA, const float2 **G, int *nsplit,
                                     int64_t *split_stride, bool *planar, cudaStream_t s, int *launches) {
    const int N = p.d.n, nb = p.d.nbins;
    *planar = false;
    if (use_pair_adjoint(p, nc)) {
        // G as fp32 [split][2 nc][N]: Re of lag l in column 2 l, Im in 2 l + 1
        const int kblocks = (p.pair_slots + 1 + 15) / 16;
        const size_t g_off = (((size_t)kblocks * 2 * nc * 128) + 1023) & ~(size_t)1023;
        Problem P{};
        P.N = N;
        P.p0 = 0;
        P.nbins = p.pair_slots + 1;
        P.ncols = 2 * nc;
        P.kblocks = kblocks;
        P.mtiles = (N + 255) / 256;
        P.ntiles = (P.ncols + TN - 1) / TN;
        const int64_t tiles = (int64_t)P.mtiles * P.ntiles;
        int ns = tiles >= p.sm_count
                     ? 1
                     : (int)std::max<int64_t>(1, std::min<int64_t>(kblocks / 16, (2LL * p.sm_count + tiles - 1) / tiles));
        ns = std::min(ns, kMaxSplit);
        while (ns > 1 && g_off + (size_t)ns * nc * N * sizeof(float2) > p.ws_alloc) --ns;
        if (g_off + (size_t)ns * nc * N * sizeof(float2) <= p.ws_alloc) {
            P.nsplit = ns;
            P.b_row0 = 0;
            P.ld = N;
            P.split_stride = (int64_t)2 * nc * N;
            P.out_off = 0;
            cudaError_t e = pack_adjoint_pair(p, dA, nc, kblocks, s);
            if (e != cudaSuccess) return e;
            *launches += 1;
            float *g = reinterpret_cast<float *>(static_cast<unsigned char *>(p.ws) + g_off);
            alignas(64) CUtensorMap omap;
            const bool tma_out = (N % 4 == 0) && p.tune_drain == 0 &&
                                 make_out_rows_map(g, N, P.ncols, ns, &omap) == cudaSuccess;
            if (adj_table(p) && p.tune_adj_atab == 2) {
                // (the G-storing contraction is bound by its epilogue: the table
                // measured 2 % slower there, so it runs with generated rows by default)
                P.a_ld = p.atab_adj_ld;
                e = launch_gemm<2, false, 2, true, true>(p, P, nullptr, nullptr, tiles * ns, g,
                                                         tma_out ? &omap : nullptr, s, p.tmap_adj);
            } else {
                e = launch_gemm<2, false, 2, true>(p, P, nullptr, nullptr, tiles * ns, g, tma_out ? &omap : nullptr, s);
            }
            if (e != cudaSuccess) return e;
            *launches += 1;
            p.last_variant = 2;
            p.last_nsplit = ns;
            p.last_tile = 256;
            *G = reinterpret_cast<const float2 *>(g);
            *nsplit = ns;
            *split_stride = (int64_t)nc * N;  // complex elements (2 nc N floats)
            *planar = true;
            return cudaSuccess;
        }
    }
    const int kblocks = (nb + 15) / 16;
    if (nc < 1 || adjoint_g_need(N, nb, nc, 1) > p.ws_alloc) return cudaErrorNotSupported;
    Problem P{};
    P.N = N;
    P.p0 = p.d.p0;
    P.nbins = nb;
    P.ncols = nc;
    P.kblocks = kblocks;
    P.mtiles = (2 * N + 255) / 256;
    P.ntiles = (nc + TN - 1) / TN;
    const int64_t tiles = (int64_t)P.mtiles * P.ntiles;
    // split the bins only while tiles are scarce (>= 16 K blocks per unit) and the splits fit
    int ns = tiles >= p.sm_count
                 ? 1
                 : (int)std::max<int64_t>(1, std::min<int64_t>(kblocks / 16, (2LL * p.sm_count + tiles - 1) / tiles));
    ns = std::min(ns, kMaxSplit);
    while (ns > 1 && adjoint_g_need(N, nb, nc, ns) > p.ws_alloc) --ns;
    P.nsplit = ns;
    P.b_row0 = 0;
    P.ld = 2LL * N;
    P.split_stride = (int64_t)nc * 2 * N;
    P.out_off = 0;
    const int64_t total = (int64_t)nc * kblocks * 16;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)p.sm_count * 16);
    k_pack_adjoint<<<blocks, 256, 0, s>>>(static_cast<const float2 *>(dA), nb, nc, kblocks,
                                          static_cast<uint2 *>(p.ws));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *launches += 1;
    float *g = reinterpret_cast<float *>(static_cast<unsigned char *>(p.ws) + adjoint_g_offset(nb, nc));
    alignas(64) CUtensorMap omap;
    const bool tma_out = (N % 2 == 0) && p.tune_drain == 0 && make_out_map(g, N, nc, ns, &omap) == cudaSuccess;
    if ((e = launch_gemm<2, false, 2>(p, P, nullptr, nullptr, tiles * ns, g, tma_out ? &omap : nullptr, s)) !=
        cudaSuccess)
        return e;
    *launches += 1;
    p.last_variant = 1;
    p.last_nsplit = ns;
    p.last_tile = 256;
    *G = reinterpret_cast<const float2 *>(g);
    *nsplit = ns;
    *split_stride = (int64_t)nc * N;  // complex elements
    return cudaSuccess;
}

// Batched CPIs: per-CPI angle tables, packed-B regions and a work list of
// (cpi, m-tile, n-tile) units, longest CPI first, built once here.  No split
// of the sample axis: the CPIs supply thousands of units.
// Largest whole-batch unpaired operand a paired batched plan keeps beside its
// two paired workspace slices (for tuning key 6 = 1).
constexpr size_t kUnpairedBatchBytes = (size_t)4 << 30;

cudaError_t ternary_batched_init(Plan &p, const ndft_cpi *cpis, int ncpi, cudaStream_t s) {
    std::vector<Problem> probs(ncpi);
    std::vector<PackProb> packs(ncpi);
    std::vector<int64_t> prefix(ncpi + 1, 0), tprefix(ncpi + 1, 0);
    int64_t ang_total = 0, rows_total = 0;
    for (int c = 0; c < ncpi; ++c) {
        const ndft_cpi &q = cpis[c];
        if (q.n > kMaxN) return cudaErrorNotSupported;
        Problem &P = probs[c];
        P.N = q.n;
        P.p0 = q.p0;
        P.nbins = q.nbins;
        P.ncols = q.nlags;
        P.kblocks = (q.n + 7) / 8;
        P.nsplit = 1;
        P.mtiles = (2 * q.nbins + 255) / 256;
        P.ntiles = (q.nlags + TN - 1) / TN;
        P.b_row0 = rows_total;
        P.out_off = 2 * q.off_out;
        P.ld = 2LL * q.nbins;
        P.split_stride = 0;
        P.nth = nth_for(q.n);
        PackProb &K = packs[c];
        K.a_off = q.off_surv;
        K.r_off = q.off_ref;
        K.N = q.n;
        K.lag0 = q.lag0;
        K.ncols = q.nlags;
        K.kblocks = P.kblocks;
        K.row0 = rows_total;
        prefix[c] = rows_total;
        rows_total += (int64_t)P.kblocks * q.nlags;
        tprefix[c + 1] = tprefix[c] + (int64_t)((P.kblocks + kPackKb - 1) / kPackKb) * ((q.nlags + 31) / 32);
        probs[c].ang = reinterpret_cast<const float2 *>(ang_total);  // offset, rebased below
        ang_total += P.nth + R_LO;
    }
    prefix[ncpi] = rows_total;
    if (rows_total >= (1LL << 31)) return cudaErrorNotSupported;  // TMA row coordinate is 32-bit
    // one output tensor map for all CPIs when they share an even nbins and every
    // surface starts on a row of 2 nbins floats
    {
        bool uniform = cpis[0].nbins % 2 == 0;
        int64_t rows = 0;
        for (int c = 0; c < ncpi && uniform; ++c) {
            const ndft_cpi &q = cpis[c];
            uniform = q.nbins == cpis[0].nbins && q.off_out % q.nbins == 0;
            rows = std::max<int64_t>(rows, q.off_out / q.nbins + q.nlags);
        }
        if (uniform && rows < (1LL << 31)) {
            p.bt_nbins = cpis[0].nbins;
            p.bt_rows = rows;
            for (int c = 0; c < ncpi; ++c) probs[c].crow0 = (int32_t)(cpis[c].off_out / cpis[c].nbins);
        }
    }
    std::vector<int> order(ncpi);
    for (int c = 0; c < ncpi; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cpis[a].n > cpis[b].n; });
    std::vector<Unit> units;
    for (int c : order)
        for (int nt = 0; nt < probs[c].ntiles; ++nt)
            for (int mt = 0; mt < probs[c].mtiles; ++mt) units.push_back(Unit{c, mt, nt, 0});
    cudaError_t e;
    float2 *ang = nullptr;
    if ((e = cudaMalloc(&ang, (size_t)ang_total * sizeof(float2))) != cudaSuccess) return e;
    p.ang = ang;
    p.table_bytes += (size_t)ang_total * sizeof(float2);
    for (int c = 0; c < ncpi; ++c) {
        const int64_t off = reinterpret_cast<int64_t>(probs[c].ang);
        probs[c].ang = ang + off;
        k_angles<<<(probs[c].nth + R_LO + 255) / 256, 256, 0, s>>>(probs[c].N, probs[c].nth, ang + off);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const BatchedLayout BL = batched_layout(ncpi, (int64_t)units.size());
    if ((e = cudaMalloc(&p.work_dev, BL.total)) != cudaSuccess) return e;
    unsigned char *wd = reinterpret_cast<unsigned char *>(p.work_dev);
    std::vector<unsigned char> host(BL.total, 0);
    std::memcpy(host.data() + BL.probs, probs.data(), probs.size() * sizeof(Problem));
    std::memcpy(host.data() + BL.packs, packs.data(), packs.size() * sizeof(PackProb));
    std::memcpy(host.data() + BL.prefix, prefix.data(), prefix.size() * sizeof(int64_t));
    std::memcpy(host.data() + BL.tprefix, tprefix.data(), tprefix.size() * sizeof(int64_t));
    std::memcpy(host.data() + BL.units, units.data(), units.size() * sizeof(Unit));
    if ((e = cudaMemcpyAsync(wd, host.data(), BL.total, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;  // `host` must outlive the copy
    p.nwork = (int64_t)units.size();
    p.b_bytes = (size_t)std::max<int64_t>(rows_total, 1) * 128;
    // the conjugate-paired calls, one CPI after another (longest first), when
    // every CPI's window pairs: regions for the largest CPI's packed B, split
    // partials and bin-0 sums
    bool pairs = true;
    std::vector<PairCpi> pc;
    int64_t bp_rows = 1;
    size_t bp_part = (size_t)4 * p.sm_count * 256 * TN * sizeof(float), bp_dc = 256;
    for (int c : order) {
        const ndft_cpi &q = cpis[c];
        const int S = pair_slots_for(q.n, q.p0, q.nbins);
        if (S < 1) {
            pairs = false;
            break;
        }
        pc.push_back(PairCpi{q.n, q.p0, q.nbins, q.lag0, q.nlags, S, q.off_surv, q.off_ref, q.off_out, probs[c].ang,
                             probs[c].nth});
        bp_rows = std::max<int64_t>(bp_rows, (int64_t)pair_kblocks(q.n) * 2 * q.nlags);
        bp_part = std::max(bp_part, (size_t)2 * q.nlags * 2 * S * sizeof(float));
        bp_dc = std::max(bp_dc, (size_t)pair_pack_tiles(q.n) * q.nlags * sizeof(float2));
    }
    size_t ws = p.b_bytes;
    p.bt_unpaired = true;
    if (pairs && bp_rows < (1LL << 31)) {
        p.bp_b_bytes = ((size_t)bp_rows * 128 + 1023) & ~(size_t)1023;
        p.bp_part_bytes = (bp_part + 1023) & ~(size_t)1023;
        p.bp_dc_bytes = (bp_dc + 1023) & ~(size_t)1023;
        // two such slices: consecutive CPIs run on the call's stream and a
        // plan-owned side stream, so one's packing and fold overlap the other's
        // contraction
        // the whole batch's unpaired operand (16 bytes per sample and lag of
        // every CPI) is kept beside them for key 6 = 1 only while it is modest
        const size_t slices = 2 * (p.bp_b_bytes + p.bp_part_bytes + p.bp_dc_bytes);
        p.bt_unpaired = p.b_bytes <= kUnpairedBatchBytes;
        ws = p.bt_unpaired ? std::max(ws, slices) : slices;
        p.pair_cpis = new (std::nothrow) PairCpi[pc.size()];
        if (!p.pair_cpis) return cudaErrorMemoryAllocation;
        std::copy(pc.begin(), pc.end(), p.pair_cpis);
        p.npair = (int32_t)pc.size();
    }
    p.ws_bytes = ws;
    p.ws_alloc = ws;
    if ((e = cudaMalloc(&p.ws, p.ws_bytes)) != cudaSuccess) return e;
    p.tmap_host = std::aligned_alloc(64, sizeof(CUtensorMap));
    if (!p.tmap_host) return cudaErrorMemoryAllocation;
    if (p.bt_unpaired &&
        (e = make_tmap(p.ws, std::max<int64_t>(rows_total, 1), static_cast<CUtensorMap *>(p.tmap_host))) !=
            cudaSuccess)
        return e;
    if (p.npair > 0) {
        const size_t slice = p.bp_b_bytes + p.bp_part_bytes + p.bp_dc_bytes;
        p.tmap_bpair = std::aligned_alloc(64, 2 * sizeof(CUtensorMap));
        if (!p.tmap_bpair) return cudaErrorMemoryAllocation;
        CUtensorMap *m = static_cast<CUtensorMap *>(p.tmap_bpair);
        if ((e = make_tmap(p.ws, bp_rows, &m[0])) != cudaSuccess) return e;
        if ((e = make_tmap(static_cast<unsigned char *>(p.ws) + slice, bp_rows, &m[1])) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithFlags(&p.side, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&p.ev_fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&p.ev_join, cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The batched plan's CPIs as conjugate-paired calls (the single-surface path
// with generated A rows): per CPI the paired packing, the contraction and the
// fold into its surface.  CPIs alternate, longest first, between the call's
// stream and the plan's side stream, each with its own workspace slice; the
// side stream forks from and joins back into the call's stream (so stream
// order and CUDA-graph capture are kept).
static cudaError_t batched_pair_calls(Plan &p, const void *surv, const void *ref, void *out, cudaStream_t s0,
                                      int *launches) {
    const bool two = p.side && p.npair > 1;
    cudaError_t e;
    if (two) {
        if ((e = cudaEventRecord(p.ev_fork, s0)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(p.side, p.ev_fork, 0)) != cudaSuccess) return e;
    }
    const bool caf = true;
    for (int k = 0; k < p.npair; ++k) {
        const int sl = two ? (k & 1) : 0;
        const cudaStream_t s = sl ? p.side : s0;
        unsigned char *ws = static_cast<unsigned char *>(p.ws) + sl * (p.bp_b_bytes + p.bp_part_bytes + p.bp_dc_bytes);
        float *part = reinterpret_cast<float *>(ws + p.bp_b_bytes);
        float2 *dc = reinterpret_cast<float2 *>(ws + p.bp_b_bytes + p.bp_part_bytes);
        const CUtensorMap *bmap = static_cast<const CUtensorMap *>(p.tmap_bpair) + sl;
        const PairCpi &q = p.pair_cpis[k];
        const int N = q.n, S = q.slots, ncols = q.nlags;
        const int kblocks = pair_kblocks(N), gy = pair_pack_tiles(N);
        PackProb pp{};
        pp.a_off = q.off_surv;
        pp.r_off = q.off_ref;
        pp.N = N;
        pp.lag0 = q.lag0;
        pp.ncols = ncols;
        pp.kblocks = kblocks;
        pp.ldx = 0;
        pp.row0 = 0;
        k_pack_pair<<<dim3((ncols + 31) / 32, std::min(gy, 65535)), 256, 0, s>>>(
            pp, p.d.flags, caf, static_cast<const float2 *>(surv), static_cast<const float2 *>(ref),
            reinterpret_cast<uint4 *>(ws), dc, gy, p.err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        Problem P{};
        P.N = N;
        P.p0 = 1;
        P.nbins = S;
        P.ncols = 2 * ncols;
        P.kblocks = kblocks;
        P.mtiles = (2 * S + 255) / 256;
        P.ntiles = (P.ncols + TN - 1) / TN;
        const int64_t tiles = (int64_t)P.mtiles * P.ntiles;
        const int64_t cap_units = (int64_t)(p.bp_part_bytes / ((size_t)256 * TN * sizeof(float)));
        P.nsplit = choose_split(tiles, kblocks, p.sm_count, p.tune_split, cap_units);
        // two CPIs share the GPU (two streams): at most 8 splits by default, which
        // keeps the partials and the fold small (measured on the 256-CPI workload:
        // 42.4 ms against 45.3 ms with one CPI's own best split count)
        if (p.tune_split == 0 && P.nsplit > 8) P.nsplit = 8;
        while (P.nsplit > 1 && (size_t)P.nsplit * P.ncols * 2 * S * sizeof(float) > p.bp_part_bytes) --P.nsplit;
        P.b_row0 = 0;
        P.ld = 2LL * S;
        P.split_stride = (int64_t)P.ncols * 2 * S;
        P.ang = q.ang;
        P.nth = q.nth;
        P.out_off = 0;
        alignas(64) CUtensorMap omap;
        const bool tma_out = (S % 2 == 0) && p.tune_drain == 0 &&
                             make_out_map(part, S, P.ncols, P.nsplit, &omap, 32) == cudaSuccess;
        if ((e = launch_gemm<2, false, 0, true>(p, P, nullptr, nullptr, tiles * P.nsplit, part,
                                                tma_out ? &omap : nullptr, s, nullptr, bmap)) != cudaSuccess)
            return e;
        const dim3 fgrid(ncols, (S + kFoldBins - 1) / kFoldBins);
        k_pair_fold<false><<<fgrid, kFoldBins, 0, s>>>(part, P.nsplit, P.split_stride, S, N, q.p0, q.nbins, dc, gy,
                                                       ncols, static_cast<float2 *>(out) + q.off_out, p.err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 3;
    }
    if (two) {
        if ((e = cudaEventRecord(p.ev_join, p.side)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s0, p.ev_join, 0)) != cudaSuccess) return e;
    }
    p.last_variant = 2;
    p.last_tile = 256;
    return cudaSuccess;
}

cudaError_t launch_ternary_batched(Plan &p, const void *surv, const void *ref, void *out, cudaStream_t s,
                                   int *launches) {
    if (p.npair > 0 && p.tune_pair != 1) return batched_pair_calls(p, surv, ref, out, s, launches);
    if (!p.bt_unpaired) return cudaErrorNotSupported;  // its operand was not kept (see the plan's set-up)
    const BatchedLayout BL = batched_layout(p.ncpi, p.nwork);
    unsigned char *wd = reinterpret_cast<unsigned char *>(p.work_dev);
    const Problem *probs = reinterpret_cast<const Problem *>(wd + BL.probs);
    const PackProb *packs = reinterpret_cast<const PackProb *>(wd + BL.packs);
    const int64_t *tprefix = reinterpret_cast<const int64_t *>(wd + BL.tprefix);
    const Unit *units = reinterpret_cast<const Unit *>(wd + BL.units);
    k_pack_tiles<<<p.sm_count * 8, 256, 0, s>>>(packs, tprefix, p.ncpi, p.d.flags, static_cast<const float2 *>(surv),
                                                static_cast<const float2 *>(ref), static_cast<uint4 *>(p.ws), p.err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *launches += 1;
    alignas(64) CUtensorMap omap;
    const bool tma_out = p.bt_rows > 0 && p.tune_drain == 0 && ((uintptr_t)out & 15u) == 0 &&
                         make_out_map(out, p.bt_nbins, (int)p.bt_rows, 1, &omap) == cudaSuccess;
    if ((e = launch_gemm<2, true>(p, Problem{}, probs, units, p.nwork, static_cast<float *>(out),
                               tma_out ? &omap : nullptr, s)) != cudaSuccess)
        return e;
    *launches += 1;
    return cudaSuccess;
}

}  // namespace ndft
