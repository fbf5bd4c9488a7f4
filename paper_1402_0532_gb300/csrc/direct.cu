// direct.cu -- the plain form: (x) evaluated term by term on the CUDA cores.
//
// Computes out[col][k] = sum_n W^((p n) mod N) (x) v[col][n], p = p0 + k, for
//   * the NDFT of Eq. 8: v = x (one column per input vector), and
//   * the nonlinear ambiguity surface of Eq. 12a: v = z_l with
//     z_l[n] = s_surv[n] (x) conj(s_ref[n - l]), one column per lag l.
//
// Each block owns 64 bins x 64 columns and walks the sample axis in chunks of
// 16.  Per chunk it stages, in shared memory, the 16 x 64 twiddles of its bins
// (gathered from the plan's fp32 table at (p n) mod N, the index advanced
// incrementally) and the 16 x 64 data values, both already split into the
// pieces (x) needs.  Each thread then accumulates a 4 x 4 register tile.
// fp32: the twiddle as magnitude and sign (a float in {-1, 0, +1}), the data
// as its signed value and sign; one real (x) accumulated is two fmas:
// fma(sgn a, fma(sgn b, |a|, b), acc) = acc + sgn(a) sgn(b)(|a| + |b|), the
// inner sum rounded once and the product by sgn a exact, so it rounds exactly
// as acc + (a (x) b) (Eq. 1-2, the zero case explicit as a zero sign).
// Q1.14: the same two fmas on exact integers.  A twiddle has |W_r| + |W_i| <=
// 2^14 sqrt 2 < 23171; a data value (int16, or the integer lag product
// z = s (x) conj(r), |z_r| + |z_i| <= 2 (|s_r| + |s_i| + |r_r| + |r_i|) <= 2^18)
// keeps sgn(b)(|a| + |b|) below 2^18 + 2^14, and one sample adds at most
// 23171 + 2^18 < 285315 to a component's sum: 48 samples (three chunks) stay
// below 2^24, so every fp32 operation is exact, and every three chunks the sums
// are converted to integers and added into int32 totals modulo 2^32 -- the
// integer (x) of Eq. 2 with wrap-around sums, bit for bit.  With NDFT_F_Q14_RANGE the totals are
// kept exact in int64 (shared memory) and a cell whose sum leaves int32 sets
// the plan's overflow code.  One complex (x) is four real ones (Eq. 6).
#include "internal.cuh"

#include <algorithm>

namespace ndft {

namespace {

constexpr int BP = 64;   // bins per block
constexpr int BC = 64;   // columns per block
constexpr int KC = 16;   // samples per chunk
constexpr int kThreads = 256;


// ---- precision traits ---------------------------------------------------------
struct PrecF32 {
    static constexpr bool kTwoLevel = true;  // see direct_tile
    static constexpr bool kIntFlush = false;
    using In = float2;
    using Tw = float2;
    using V = float2;
    using Mag = float2;
    using Sgn = float2;  // sgn(v.x), sgn(v.y) in {-1, 0, +1}
    using Acc = float2;
    __device__ static V load(const In *p, int64_t i) { return p[i]; }
    __device__ static V zero() { return make_float2(0.f, 0.f); }
    __device__ static V conj_(V v) { return make_float2(v.x, -v.y); }
    __device__ static V cox(V a, V b) { return cox_f32(a, b); }
    __device__ static float sgn1(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }
    // twiddle side: magnitudes and signs
    __device__ static void ready(V v, Mag &m, Sgn &s) {
        m = make_float2(fabsf(v.x), fabsf(v.y));
        s = make_float2(sgn1(v.x), sgn1(v.y));
    }
    // data side: the signed value itself and its sign
    __device__ static void ready_data(V v, Mag &m, Sgn &s) {
        m = v;
        s = make_float2(sgn1(v.x), sgn1(v.y));
    }
    __device__ static Acc acc0() { return make_float2(0.f, 0.f); }
    // acc += w (x) v, Eq. 6: re += w_r(x)v_r - w_i(x)v_i, im += w_i(x)v_r + v_i(x)w_r.
    // Each a (x) b with a the twiddle component and b the data component is
    // fma(sgn a, fma(sgn b, |a|, b), acc): the inner fma is sgn(b)(|a| + |b|)
    // rounded once (round to nearest is symmetric; 0 when b = 0), the outer
    // scales it exactly by sgn a (0 when a = 0) and rounds the sum once, so the
    // result is fl(acc + a (x) b) with a (x) b rounded once (Eq. 1): two
    // instructions per real (x).  wm, ws: |w|, sgn w; vv, vs: v, sgn v.
    __device__ static void mac(Acc &acc, const Mag &wm, const Sgn &ws, const Mag &vv, const Sgn &vs) {
        acc.x = __fmaf_rn(ws.x, __fmaf_rn(vs.x, wm.x, vv.x), acc.x);
        acc.x = __fmaf_rn(-ws.y, __fmaf_rn(vs.y, wm.y, vv.y), acc.x);
        acc.y = __fmaf_rn(ws.y, __fmaf_rn(vs.x, wm.y, vv.x), acc.y);
        acc.y = __fmaf_rn(ws.x, __fmaf_rn(vs.y, wm.x, vv.y), acc.y);
    }
    using Out = float2;
};

struct PrecQ14 {
    static constexpr bool kTwoLevel = false;
    static constexpr bool kIntFlush = true;  // exact fp32 chunk sums -> int32 totals (wrap)
    using In = short2;
    using Tw = short2;
    using V = int2;
    using Mag = float2;  // twiddle: |w|; data: the value itself (exact integers)
    using Sgn = float2;  // signs in {-1, 0, +1}
    using Acc = float2;  // one chunk's sums, exact integers < 2^24
    __device__ static V load(const In *p, int64_t i) {
        const short2 v = p[i];
        return make_int2(v.x, v.y);
    }
    __device__ static V zero() { return make_int2(0, 0); }
    __device__ static V conj_(V v) { return make_int2(v.x, -v.y); }
    __device__ static V cox(V a, V b) { return cox_i32(a, b); }
    __device__ static float sgn1(int v) { return v > 0 ? 1.f : (v < 0 ? -1.f : 0.f); }
    // exact int -> float for |v| < 2^22 on the integer and fp32 pipes: the bits
    // v + 0x4B400000 are the float 1.5 2^23 + v (the conversion instruction
    // runs on a quarter-rate pipe)
    __device__ static float i2f(int v) { return __int_as_float(v + 0x4B400000) - 12582912.0f; }
    __device__ static void ready(V v, Mag &m, Sgn &s) {
        m = make_float2(i2f(abs(v.x)), i2f(abs(v.y)));
        s = make_float2(sgn1(v.x), sgn1(v.y));
    }
    __device__ static void ready_data(V v, Mag &m, Sgn &s) {
        m = make_float2(i2f(v.x), i2f(v.y));
        s = make_float2(sgn1(v.x), sgn1(v.y));
    }
    __device__ static Acc acc0() { return make_float2(0.f, 0.f); }
    __device__ static void mac(Acc &acc, const Mag &wm, const Sgn &ws, const Mag &vv, const Sgn &vs) {
        PrecF32::mac(acc, wm, ws, vv, vs);
    }
    using Out = uint2;
};

template <class P>
__device__ __forceinline__ typename P::V load_tw(const typename P::Tw *tw, int64_t m) {
    return P::load(tw, m);
}

// ---- data sources ------------------------------------------------------------
template <class P>
struct NdftSrc {
    const typename P::In *x;
    int64_t ld;  // row stride (= N)
    __device__ typename P::V operator()(int64_t col, int64_t n) const { return P::load(x, col * ld + n); }
};

template <class P>
struct CafSrc {
    const typename P::In *ss;
    const typename P::In *sr;
    int N;
    int lag0;
    uint32_t flags;
    __device__ typename P::V operator()(int64_t col, int64_t n) const {
        int64_t j = n - (lag0 + col);
        typename P::V ref = P::zero();
        if (flags & NDFT_F_CIRCULAR_LAG) {
            j %= N;
            if (j < 0) j += N;
        }
        if (j >= 0 && j < N) {
            ref = P::load(sr, j);
            if (!(flags & NDFT_F_NO_CONJ_REF)) ref = P::conj_(ref);
        }
        return P::cox(P::load(ss, n), ref);  // lag product of Eq. 12a
    }
};

struct Smem {
    // [KC][BP + 2] magnitudes (fp32 data: values) and [KC][BP + 1] sign/zero words, twiddles then data.
    static constexpr int kMagStride = BP + 2;
    static constexpr int kSgnStride = BP + 1;
    __host__ __device__ static constexpr size_t bytes(size_t mag_size, size_t sgn_size) {
        return 2 * (KC * kMagStride * mag_size + KC * kSgnStride * sgn_size);
    }
    // fp32: each thread's 16 outer accumulators [cell][thread] after the staging
    static constexpr size_t kOuter = 16 * kThreads * sizeof(float2);
    // Q1.14 with the range check: each thread's 16 exact int64 totals (Re, Im) [2 cell + c][thread]
    static constexpr size_t kTot64 = 32 * kThreads * sizeof(long long);
    template <class P, bool CHK = false>
    static constexpr size_t bytes_for() {
        return bytes(sizeof(typename P::Mag), sizeof(typename P::Sgn)) + (P::kTwoLevel ? kOuter : 0) +
               (CHK ? kTot64 : 0);
    }
};

// Q1.14: chunks per exact fp32 partial sum (see the bound above)
constexpr int kIntFlushChunks = 3;

// fp32 sums run in two levels: the register accumulators take kFlushChunks
// chunks (1024 samples) and are then added into per-thread outer sums in
// shared memory, so no single fp32 running sum takes more than
// max(1024, N / 1024) terms (a single level over 2^20 incoherent terms
// exceeded 1e-5 of max|X|).
constexpr int kFlushChunks = 64;

// One 64 x 64 tile over samples [n_begin, n_end).  out points at the tile's
// [col][bin] destination with row stride ldo.
template <class P, class Src, bool CHK = false>
__device__ __forceinline__ void direct_tile(unsigned char *smem, const typename P::Tw *__restrict__ tw, int N,
                                            int p0, int nbins, int ncols, int bin0, int col0, int64_t n_begin,
                                            int64_t n_end, const Src &src, typename P::Out *__restrict__ out,
                                            int64_t ldo, int32_t *err) {
    static_assert(!CHK || P::kIntFlush, "the range check is for the integer form");
    using Mag = typename P::Mag;
    Mag *tM = reinterpret_cast<Mag *>(smem);
    using Sgn = typename P::Sgn;
    Sgn *tS = reinterpret_cast<Sgn *>(tM + KC * Smem::kMagStride);
    Mag *vM = reinterpret_cast<Mag *>(tS + KC * Smem::kSgnStride);
    Sgn *vS = reinterpret_cast<Sgn *>(vM + KC * Smem::kMagStride);

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    // twiddle staging: fixed bin b, samples kk = (tid >> 6) + 4 j
    const int sb = tid & 63;
    const int bin = bin0 + sb;
    const bool bin_ok = bin < nbins;
    int64_t pm = ((int64_t)p0 + bin) % N;
    if (pm < 0) pm += N;
    int64_t m[4];
    const int kk0 = tid >> 6;
#pragma unroll
    for (int j = 0; j < 4; ++j) m[j] = (pm * ((n_begin + kk0 + 4 * j) % N)) % N;
    const int64_t step = (pm * KC) % N;

    // data staging: fixed sample kk = tid & 15, columns c = (tid >> 4) + 16 j
    const int dk = tid & 15, dc0 = tid >> 4;

    typename P::Acc acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = P::acc0();
    // outer sums: only this thread touches its 16 entries, so no barrier is needed
    float2 *outer = reinterpret_cast<float2 *>(smem + Smem::bytes(sizeof(Mag), sizeof(Sgn)));
    if constexpr (P::kTwoLevel) {
#pragma unroll
        for (int c = 0; c < 16; ++c) outer[c * kThreads + tid] = make_float2(0.f, 0.f);
    }
    // integer form: int32 totals modulo 2^32, or exact int64 totals in shared memory (CHK)
    uint2 tot[4][4];
    long long *tot64 = reinterpret_cast<long long *>(smem + Smem::bytes(sizeof(Mag), sizeof(Sgn)));
    if constexpr (P::kIntFlush) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) tot[i][j] = make_uint2(0u, 0u);
        if constexpr (CHK) {
#pragma unroll
            for (int c = 0; c < 32; ++c) tot64[c * kThreads + tid] = 0;
        }
    }
    int chunk_count = 0;

    for (int64_t n0 = n_begin; n0 < n_end; n0 += KC) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int kk = kk0 + 4 * j;
            const bool ok = bin_ok && (n0 + kk < n_end);
            typename P::V w = ok ? load_tw<P>(tw, m[j]) : P::zero();
            Mag mg;
            Sgn sg;
            P::ready(w, mg, sg);
            tM[kk * Smem::kMagStride + sb] = mg;
            tS[kk * Smem::kSgnStride + sb] = sg;
            m[j] += step;
            if (m[j] >= N) m[j] -= N;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = dc0 + 16 * j;
            const int64_t n = n0 + dk;
            typename P::V v = (n < n_end && col0 + c < ncols) ? src(col0 + c, n) : P::zero();
            Mag mg;
            Sgn sg;
            P::ready_data(v, mg, sg);
            vM[dk * Smem::kMagStride + c] = mg;
            vS[dk * Smem::kSgnStride + c] = sg;
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < KC; ++kk) {
            Mag wm[4], vm[4];
            Sgn ws[4], vs[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                // bins ty*4 + i: two distinct per warp (broadcast); columns tx + 16 i:
                // consecutive across the warp's 16 distinct tx, conflict-free
                wm[i] = tM[kk * Smem::kMagStride + ty * 4 + i];
                ws[i] = tS[kk * Smem::kSgnStride + ty * 4 + i];
                vm[i] = vM[kk * Smem::kMagStride + tx + 16 * i];
                vs[i] = vS[kk * Smem::kSgnStride + tx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) P::mac(acc[i][j], wm[i], ws[i], vm[j], vs[j]);
        }
        __syncthreads();
        if constexpr (P::kIntFlush) {
            // every kIntFlushChunks chunks (and after the last) the exact integer
            // sums (< 2^24 in magnitude) into the totals
            if (++chunk_count == kIntFlushChunks || n0 + KC >= n_end) {
            chunk_count = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int rx = __float2int_rn(acc[i][j].x), ry = __float2int_rn(acc[i][j].y);
                    if constexpr (CHK) {
                        tot64[(2 * (i * 4 + j)) * kThreads + tid] += rx;
                        tot64[(2 * (i * 4 + j) + 1) * kThreads + tid] += ry;
                    } else {
                        tot[i][j].x += (uint32_t)rx;
                        tot[i][j].y += (uint32_t)ry;
                    }
                    acc[i][j] = P::acc0();
                }
            }
        }
        if constexpr (P::kTwoLevel) {
            if (++chunk_count == kFlushChunks) {
                chunk_count = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float2 &o = outer[(i * 4 + j) * kThreads + tid];
                        o = make_float2(__fadd_rn(o.x, acc[i][j].x), __fadd_rn(o.y, acc[i][j].y));
                        acc[i][j] = P::acc0();
                    }
            }
        }
    }
    if constexpr (P::kTwoLevel) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 o = outer[(i * 4 + j) * kThreads + tid];
                acc[i][j] = make_float2(__fadd_rn(o.x, acc[i][j].x), __fadd_rn(o.y, acc[i][j].y));
            }
    }

    if constexpr (CHK) {
        bool wrapped = false;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long vx = tot64[(2 * (i * 4 + j)) * kThreads + tid];
                const long long vy = tot64[(2 * (i * 4 + j) + 1) * kThreads + tid];
                const bool live = (col0 + tx + 16 * j < ncols) && (bin0 + ty * 4 + i < nbins);
                wrapped |= live && (vx != (long long)(int32_t)vx || vy != (long long)(int32_t)vy);
                tot[i][j] = make_uint2((uint32_t)(unsigned long long)vx, (uint32_t)(unsigned long long)vy);
            }
        if (wrapped) dev_set_error(err, kDevOverflow);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = col0 + tx + 16 * j;
        if (col >= ncols) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int b = bin0 + ty * 4 + i;
            if (b < nbins && ndft_in(ldo >= nbins, err)) {
                if constexpr (P::kIntFlush) out[(int64_t)col * ldo + b] = tot[i][j];
                else out[(int64_t)col * ldo + b] = acc[i][j];
            }
        }
    }
}

template <class P, class Src, bool CHK = false>
__global__ void __launch_bounds__(kThreads, 2)
    k_direct(const typename P::Tw *__restrict__ tw, int N, int p0, int nbins, int ncols, Src src,
             int64_t samples_per_split, typename P::Out *__restrict__ out, int32_t *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int bin0 = blockIdx.x * BP;
    const int col0 = blockIdx.y * BC;
    const int64_t n_begin = (int64_t)blockIdx.z * samples_per_split;
    const int64_t n_end = min((int64_t)N, n_begin + samples_per_split);
    typename P::Out *o = out + (int64_t)blockIdx.z * ncols * nbins;
    direct_tile<P, Src, CHK>(smem, tw, N, p0, nbins, ncols, bin0, col0, n_begin, n_end, src, o, nbins, err);
}

// Persistent kernel over the CPI work list of a batched plan.  Unit u of the
// list encodes (cpi, bin tile, lag tile); units are fetched with an atomic
// counter, longest CPIs first, and each writes its tile of that CPI's surface.
template <class P, bool CHK = false>
__global__ void __launch_bounds__(kThreads, 2)
    k_direct_batched(const CpiDev *__restrict__ cpis, const int32_t *__restrict__ work, int64_t nwork,
                     int32_t *__restrict__ counter, const unsigned char *__restrict__ tab_arena,
                     const typename P::In *__restrict__ surv, const typename P::In *__restrict__ ref,
                     typename P::Out *__restrict__ outb, uint32_t flags, int32_t *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t s_unit;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int32_t u = s_unit;
        __syncthreads();
        if (u >= nwork) break;
        const int32_t c = work[3 * u], bt = work[3 * u + 1], lt = work[3 * u + 2];
        const CpiDev cp = cpis[c];
        const typename P::Tw *tw = reinterpret_cast<const typename P::Tw *>(tab_arena) + cp.tw_off;
        CafSrc<P> src{surv + cp.off_surv, ref + cp.off_ref, cp.n, cp.lag0, flags};
        direct_tile<P, CafSrc<P>, CHK>(smem, tw, cp.n, cp.p0, cp.nbins, cp.nlags, bt * BP, lt * BC, 0, cp.n,
                                       src, outb + cp.off_out, cp.nbins, err);
    }
}

template <class K>
cudaError_t prep_kernel(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

// Splits of the sample axis: the count in [1, 16] (and at most N / 64, four
// 16-sample chunks per block) whose blocks fill the resident slots (2 blocks
// per SM) in the best-quantised waves; the smallest such count when several
// are within 1 %.  Small problems (few tiles) split most: a block runs its
// samples one after another.
int direct_caf_splits(int N, int nlags, int nbins, int sm_count, int tune) {
    if (tune > 0) return std::max(1, std::min(tune, std::max(1, N / KC)));
    const int64_t tiles = (int64_t)((nbins + BP - 1) / BP) * ((nlags + BC - 1) / BC);
    const int64_t slots = 2LL * sm_count;
    const int cap = std::max(1, std::min(16, N / (4 * KC)));
    int best_s = 1;
    double best = -1.0;
    for (int c = 1; c <= cap; ++c) {
        const int64_t blocks = tiles * c;
        const double eff = (double)blocks / (double)(((blocks + slots - 1) / slots) * slots);
        if (eff > best + 0.01) {
            best = eff;
            best_s = c;
        }
    }
    return best_s;
}

// NDFT calls split their sample axis only while the partials fit in this
// much of the workspace (a split pays off only for calls of few tiles).
constexpr size_t kNdftSplitBytes = (size_t)32 << 20;

size_t direct_ws_bytes(const ndft_desc &d, int sm_count) {
    const int nb = d.nbins ? d.nbins : d.n;
    const int s = 16;  // upper bound of direct_caf_splits
    (void)sm_count;
    size_t b = 0;
    if (d.max_lags > 0) b = (size_t)s * d.max_lags * nb * sizeof(float2);
    if (d.max_batch > 0) b = std::max(b, std::min((size_t)s * d.max_batch * nb * sizeof(float2), kNdftSplitBytes));
    return b;
}

cudaError_t launch_direct_ndft(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s,
                               int *launches) {
    const int N = p.d.n, nb = p.d.nbins ? p.d.nbins : N;
    if (batch == 0) return cudaSuccess;
    const bool chk = p.d.prec == NDFT_PREC_Q14 && (p.d.flags & NDFT_F_Q14_RANGE);
    // split the sample axis like the CAF when the call has few tiles and the
    // partials fit the workspace (the range check needs whole sums: no split)
    int nsplit = chk || batch > INT32_MAX ? 1 : direct_caf_splits(N, (int)batch, nb, p.sm_count, p.tune_split);
    while (nsplit > 1 && (size_t)nsplit * batch * nb * sizeof(float2) > p.ws_alloc) --nsplit;
    const int64_t per = ((int64_t)N + nsplit - 1) / nsplit;
    const int64_t per_al = ((per + KC - 1) / KC) * KC;
    const int ns = (int)((N + per_al - 1) / per_al);
    dim3 grid((nb + BP - 1) / BP, (unsigned)((batch + BC - 1) / BC), ns);
    if (grid.y > 65535) return cudaErrorInvalidConfiguration;
    const bool split = ns > 1;
    cudaError_t e;
    if (p.d.prec == NDFT_PREC_FP32) {
        const size_t sm = Smem::bytes_for<PrecF32>();
        auto k = k_direct<PrecF32, NdftSrc<PrecF32>>;
        if ((e = prep_kernel(k, sm)) != cudaSuccess) return e;
        float2 *dst = split ? static_cast<float2 *>(p.ws) : static_cast<float2 *>(X);
        timer_begin(p, s);
        k<<<grid, kThreads, sm, s>>>(p.tw32, N, p.d.p0, nb, (int)batch,
                                     NdftSrc<PrecF32>{static_cast<const float2 *>(x), N}, per_al, dst, p.err);
        timer_end(p, s);
    } else if (chk) {
        const size_t sm = Smem::bytes_for<PrecQ14, true>();
        auto k = k_direct<PrecQ14, NdftSrc<PrecQ14>, true>;
        if ((e = prep_kernel(k, sm)) != cudaSuccess) return e;
        timer_begin(p, s);
        k<<<grid, kThreads, sm, s>>>(p.twq, N, p.d.p0, nb, (int)batch,
                                     NdftSrc<PrecQ14>{static_cast<const short2 *>(x), N}, per_al,
                                     static_cast<uint2 *>(X), p.err);
        timer_end(p, s);
    } else {
        const size_t sm = Smem::bytes_for<PrecQ14>();
        auto k = k_direct<PrecQ14, NdftSrc<PrecQ14>>;
        if ((e = prep_kernel(k, sm)) != cudaSuccess) return e;
        uint2 *dst = split ? static_cast<uint2 *>(p.ws) : static_cast<uint2 *>(X);
        timer_begin(p, s);
        k<<<grid, kThreads, sm, s>>>(p.twq, N, p.d.p0, nb, (int)batch,
                                     NdftSrc<PrecQ14>{static_cast<const short2 *>(x), N}, per_al, dst, p.err);
        timer_end(p, s);
    }
    *launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (split) {
        *launches += 1;
        if (p.d.prec == NDFT_PREC_FP32)
            return launch_reduce_splits(static_cast<const float *>(p.ws), ns, batch * nb * 2, static_cast<float *>(X),
                                        s);
        return launch_reduce_splits_i32(static_cast<const uint32_t *>(p.ws), ns, batch * nb * 2,
                                        static_cast<uint32_t *>(X), s);
    }
    return cudaSuccess;
}

cudaError_t direct_caf_preload() {
    auto k = k_direct<PrecF32, CafSrc<PrecF32>>;
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k);
    if (e != cudaSuccess) return e;
    return prep_kernel(k, Smem::bytes_for<PrecF32>());
}

cudaError_t launch_direct_caf(const Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags,
                              void *A, cudaStream_t s, int *launches) {
    const int N = p.d.n, nb = p.d.nbins ? p.d.nbins : N;
    const bool chk = p.d.prec == NDFT_PREC_Q14 && (p.d.flags & NDFT_F_Q14_RANGE);
    // the range check needs every cell's whole sum in one block: no split
    const int nsplit = chk ? 1 : direct_caf_splits(N, nlags, nb, p.sm_count, p.tune_split);
    const int64_t per = ((int64_t)N + nsplit - 1) / nsplit;
    const int64_t per_al = ((per + KC - 1) / KC) * KC;
    const int ns = (int)((N + per_al - 1) / per_al);
    dim3 grid((nb + BP - 1) / BP, (nlags + BC - 1) / BC, ns);
    cudaError_t e;
    const bool abs_out = (p.d.flags & NDFT_F_ABS_OUT) != 0;
    const bool direct_out = (ns == 1) && !abs_out;  // |A| is formed by the split sum
    if (p.d.prec == NDFT_PREC_FP32) {
        const size_t sm = Smem::bytes_for<PrecF32>();
        auto k = k_direct<PrecF32, CafSrc<PrecF32>>;
        if ((e = prep_kernel(k, sm)) != cudaSuccess) return e;
        float2 *dst = direct_out ? static_cast<float2 *>(A) : static_cast<float2 *>(p.ws);
        CafSrc<PrecF32> src{static_cast<const float2 *>(s_surv), static_cast<const float2 *>(s_ref), N, lag0,
                            p.d.flags};
        timer_begin(p, s);
        k<<<grid, kThreads, sm, s>>>(p.tw32, N, p.d.p0, nb, nlags, src, per_al, dst, p.err);
        timer_end(p, s);
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (!direct_out) {
            *launches += 1;
            if (abs_out)
                return launch_reduce_abs(static_cast<const float2 *>(p.ws), ns, (int64_t)nlags * nb,
                                         static_cast<float *>(A), s);
            return launch_reduce_splits(static_cast<const float *>(p.ws), ns, (int64_t)nlags * nb * 2,
                                        static_cast<float *>(A), s);
        }
    } else {
        uint2 *dst = direct_out ? static_cast<uint2 *>(A) : static_cast<uint2 *>(p.ws);
        CafSrc<PrecQ14> src{static_cast<const short2 *>(s_surv), static_cast<const short2 *>(s_ref), N, lag0,
                            p.d.flags};
        if (chk) {
            const size_t sm = Smem::bytes_for<PrecQ14, true>();
            auto k = k_direct<PrecQ14, CafSrc<PrecQ14>, true>;
            if ((e = prep_kernel(k, sm)) != cudaSuccess) return e;
            timer_begin(p, s);
            k<<<grid, kThreads, sm, s>>>(p.twq, N, p.d.p0, nb, nlags, src, per_al, dst, p.err);
            timer_end(p, s);
        } else {
            const size_t sm = Smem::bytes_for<PrecQ14>();
            auto k = k_direct<PrecQ14, CafSrc<PrecQ14>>;
            if ((e = prep_kernel(k, sm)) != cudaSuccess) return e;
            timer_begin(p, s);
            k<<<grid, kThreads, sm, s>>>(p.twq, N, p.d.p0, nb, nlags, src, per_al, dst, p.err);
            timer_end(p, s);
        }
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (!direct_out) {
            *launches += 1;
            return launch_reduce_splits_i32(static_cast<const uint32_t *>(p.ws), ns, (int64_t)nlags * nb * 2,
                                            static_cast<uint32_t *>(A), s);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_direct_batched(const Plan &p, const void *surv, const void *ref, void *out, cudaStream_t s,
                                  int *launches) {
    cudaError_t e = cudaMemsetAsync(p.counter, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int grid = p.sm_count * 2;
    if (p.d.prec == NDFT_PREC_FP32) {
        const size_t sm = Smem::bytes_for<PrecF32>();
        auto k = k_direct_batched<PrecF32>;
        if ((e = prep_kernel(k, sm)) != cudaSuccess) return e;
        timer_begin(p, s);
        k<<<grid, kThreads, sm, s>>>(p.cpis_dev, p.work_dev, p.nwork, p.counter,
                                     static_cast<const unsigned char *>(p.tab_arena),
                                     static_cast<const float2 *>(surv), static_cast<const float2 *>(ref),
                                     static_cast<float2 *>(out), p.d.flags, p.err);
        timer_end(p, s);
    } else if (p.d.flags & NDFT_F_Q14_RANGE) {
        const size_t sm = Smem::bytes_for<PrecQ14, true>();
        auto k = k_direct_batched<PrecQ14, true>;
        if ((e = prep_kernel(k, sm)) != cudaSuccess) return e;
        timer_begin(p, s);
        k<<<grid, kThreads, sm, s>>>(p.cpis_dev, p.work_dev, p.nwork, p.counter,
                                     static_cast<const unsigned char *>(p.tab_arena),
                                     static_cast<const short2 *>(surv), static_cast<const short2 *>(ref),
                                     static_cast<uint2 *>(out), p.d.flags, p.err);
        timer_end(p, s);
    } else {
        const size_t sm = Smem::bytes_for<PrecQ14>();
        auto k = k_direct_batched<PrecQ14>;
        if ((e = prep_kernel(k, sm)) != cudaSuccess) return e;
        timer_begin(p, s);
        k<<<grid, kThreads, sm, s>>>(p.cpis_dev, p.work_dev, p.nwork, p.counter,
                                     static_cast<const unsigned char *>(p.tab_arena),
                                     static_cast<const short2 *>(surv), static_cast<const short2 *>(ref),
                                     static_cast<uint2 *>(out), p.d.flags, p.err);
        timer_end(p, s);
    }
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace ndft
