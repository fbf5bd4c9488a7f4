// internal.cuh -- plan object, device helpers and launcher declarations shared
// by the library's translation units.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/ndft.h"

namespace ndft {

constexpr uint32_t kSignBit = 0x80000000u;

// The lag window lag0 .. lag0 + nlags - 1 of a CAF call must be representable
// in int32 so that every per-lag index (lag0 + a) is an int without overflow.
inline bool lag_window_ok(int32_t lag0, int32_t nlags) {
    return nlags >= 1 && (int64_t)lag0 + nlags - 1 <= (int64_t)INT32_MAX;
}

// Device error codes written to the plan's error word (first writer wins).
enum DevErr : int32_t { kDevOk = 0, kDevTimeout = 5, kDevOverflow = 6, kDevBadIndex = 7 };

// One CPI of a batched plan, as the kernels see it (device copy).
struct CpiDev {
    int64_t off_surv, off_ref, off_out;
    int32_t n, lag0, nlags, p0, nbins;
    int32_t tab;        // index of this CPI's twiddle tables in the table arena
    int64_t tw_off;     // element offset of its fp32 / Q1.14 full table
    int64_t qt_off;     // element offset of its bf16 quarter table
    int64_t b_off;      // element offset (bf16) of its packed B operand in the workspace
    int64_t ws_off;     // element offset (float) of its split-K partials
    int32_t nsplit;     // sample-axis splits
    int32_t kblocks;    // 64-wide K blocks (ternary form)
};

// One CPI of a batched tensor-core plan, for its conjugate-paired call.
struct PairCpi {
    int32_t n, p0, nbins, lag0, nlags, slots;
    int64_t off_surv, off_ref, off_out;  // elements from the call's bases
    const float2 *ang;                   // its two-level (cos, sin) table
    int32_t nth;
};

struct Plan {
    ndft_desc d{};
    bool batched = false;
    int device = 0;
    int sm_count = 0;
    int g4 = 1;                  // gcd(4, N)
    // tables (single-CPI plans)
    float2 *tw32 = nullptr;      // [N]
    short2 *twq = nullptr;       // [N]
    float2 *ang = nullptr;       // ternary form: two-level (cos, sin) table
    float2 *nfft_ws = nullptr;   // 8192 <= N <= 65536: intermediate of the two-kernel NFFT
    int64_t nfft_chunk = 0;      // vectors per pass through nfft_ws
    float2 *comb = nullptr;      // 2N: comb-major copies of s_surv, s_ref (two-kernel DIT CAF)
    // workspace
    void *ws = nullptr;
    size_t ws_alloc = 0;         // bytes of ws itself
    size_t ws_bytes = 0;         // every workspace buffer of the plan
    int32_t *err = nullptr;      // device error word
    size_t table_bytes = 0;
    // batched
    int32_t ncpi = 0;
    CpiDev *cpis_dev = nullptr;
    CpiDev *cpis_host = nullptr;
    void *tab_arena = nullptr;   // per-CPI tables
    int32_t *work_dev = nullptr; // work list (ternary / direct units)
    int64_t nwork = 0;
    int32_t *counter = nullptr;  // persistent-kernel tile counter
    // tuning
    int tune_split = 0;
    int tune_cols = 0;
    int tune_chunk = 0;          // ternary form: K blocks per TMEM accumulation chain
    int tune_drain = 0;          // ternary form: 0 bulk tensor stores/adds, 1 per-element adds
    int test_starve = 0;         // ternary form, tests only: issue no operand loads (waits run out)
    int tune_parts = 1;          // ternary form: 1 one part (default); 0 two parts, half each; else part 0's columns
    int tune_pair = 0;           // ternary form: 0 conjugate-paired rows where they save work (default), 1 never
    int pair_slots = 0;          // ternary form: frequencies 1 .. pair_slots cover the bin window (0: none)
    int tune_look = 0;           // items the in-tile packers run ahead (0: 4)
    int tune_bgen = 0;           // paired B operand on the pair tile: 0/3 packed just in time by its own warps,
                                 // 1 packed by a kernel before it, 2 formed in its shared memory
    int tune_atab = 0;           // ternary form: 0 paired A tiles from the plan's table when built, 1 generated on chip
    void *atab = nullptr;        // ternary form: the paired contraction's A operand, [K block][rows] x 128 B
    size_t atab_bytes = 0;
    int32_t atab_ld = 0;         // its rows per K block
    void *tmap_a = nullptr;      // its TMA descriptor (host copy)
    void *tmap_a2 = nullptr;     // the same with a 128-row box (2-SM pair tile)
    void *atab_adj = nullptr;    // ternary CAF plans: the paired adjoint's sign rows
    size_t atab_adj_bytes = 0;
    int32_t atab_adj_ld = 0;     // its rows per K block (samples padded to 256)
    void *tmap_adj = nullptr;    // its TMA descriptor (host copy)
    int tune_adj_atab = 0;       // the adjoint's A tiles from that table: 0 for dL/ds_surv, 2 for both, 1 neither
    size_t dc_bytes = 0;         // ternary form: per-tile DC sums of the paired packing, then item flags
    size_t dc_flag_off = 0;      // offset of the item flags in that region
    // ternary form: side stream and events of the two-part contraction (the
    // second part's packing runs under the first part's contraction)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int last_launches = 0;
    int last_variant = 0;        // contraction of the last exec call: 0 none, 1 unpaired rows, 2 paired rows
    int last_nsplit = 0;         // its sample-axis split count
    int last_tile = 0;           // its tile: 256 / 128 rows on one CTA, 258 the 2-SM pair
    // optional timing of the main contraction kernel (event pairs, see ndft_timer_start)
    mutable cudaEvent_t *tev = nullptr;
    mutable int tcap = 0;
    mutable int tcount = 0;
    // ternary GEMM: TMA descriptor storage (host copy + device copy)
    void *tmap_host = nullptr;
    void *tmap_host2 = nullptr;  // same buffer, 128-row box (one CTA's half of B in the pair tile)
    void *tmap_dev = nullptr;
    size_t b_bytes = 0;          // packed-B region of the workspace
    size_t part_bytes = 0;       // split-K partials region of the workspace
    // batched ternary plans: the output viewed as one [rows][2 nbins] fp32 tensor
    // for the bulk-copy fold-out (0 rows: CPIs differ in nbins or are not row-aligned)
    PairCpi *pair_cpis = nullptr;  // batched tensor-core plans: the CPIs, longest first, when all pair
    int32_t npair = 0;
    size_t bp_b_bytes = 0, bp_part_bytes = 0, bp_dc_bytes = 0;  // their workspace regions
    void *tmap_bpair = nullptr;    // TMA descriptors of their packed B regions (two slices)
    bool bt_unpaired = true;       // the whole batch's unpaired operand fits the workspace
    int32_t bt_nbins = 0;
    int64_t bt_rows = 0;
};

// ---- the operator on device ------------------------------------------------------

// sgn(v) in two instructions: 1.0f where v != 0 (set.ne), with v's sign bit
// copied in, so +-1, or a zero of v's sign for a zero v.  As a factor it is
// exact; a zero of either sign contributes nothing to a nonzero sum.
__device__ __forceinline__ float sgn_mul(float v) {
    float nz;
    asm("set.ne.f32.f32 %0, %1, 0f00000000;" : "=f"(nz) : "f"(v));
    return __uint_as_float(__float_as_uint(nz) | (__float_as_uint(v) & kSignBit));
}

// Eq. 6 on raw fp32 values: (a_r (x) b_r - a_i (x) b_i, a_i (x) b_r + a_r (x) b_i),
// each real (x) rounded once (Eq. 1-2), then one subtraction / addition.  A
// real a (x) b = sgn(a) sgn(b) (|a| + |b|) starts as the inner
// fma(sgn b, |a|, b) = sgn(b) (|a| + |b|), rounded once (round to nearest is
// sign-symmetric); scaling it by sgn a (+-1 or a zero) is exact, so the
// difference and the sum take one fma each, whose addend is the other term
// scaled by one more fma with a +0 addend.  Every addend is then nonzero or
// +0, so no fma returns -0: a zero result is +0, as the definition's 0 for a
// zero operand and as an exactly cancelling difference.  The same bits as
// rounding |a| + |b| with the XOR of the sign bits per term and combining the
// terms one by one, in 18 instructions instead of about 26.
__device__ __forceinline__ float2 cox_f32(float2 a, float2 b) {
    const float sar = sgn_mul(a.x), sai = sgn_mul(a.y), sbr = sgn_mul(b.x), sbi = sgn_mul(b.y);
    const float i1 = __fmaf_rn(sbr, fabsf(a.x), b.x);  // sgn b_r (|a_r| + |b_r|)
    const float i2 = __fmaf_rn(sbi, fabsf(a.y), b.y);  // sgn b_i (|a_i| + |b_i|)
    const float i3 = __fmaf_rn(sbr, fabsf(a.y), b.x);  // sgn b_r (|a_i| + |b_r|)
    const float i4 = __fmaf_rn(sbi, fabsf(a.x), b.y);  // sgn b_i (|a_r| + |b_i|)
    const float n2 = __fmaf_rn(-sai, i2, 0.f);         // -(a_i (x) b_i)
    const float t4 = __fmaf_rn(sar, i4, 0.f);          // a_r (x) b_i
    return make_float2(__fmaf_rn(sar, i1, n2), __fmaf_rn(sai, i3, t4));
}

// Integer (x) (Q1.14 units): sgn(a) sgn(b) (|a| + |b|), 0 if either is 0.
__device__ __forceinline__ int32_t ox_i32(int32_t a, int32_t b) {
    int32_t m = abs(a) + abs(b);
    int32_t s = (a ^ b) >> 31;             // -1 if the signs differ
    int32_t r = (m ^ s) - s;
    return (a != 0 && b != 0) ? r : 0;
}

__device__ __forceinline__ int2 cox_i32(int2 a, int2 b) {
    return make_int2(ox_i32(a.x, b.x) - ox_i32(a.y, b.y), ox_i32(a.y, b.x) + ox_i32(b.y, a.x));
}

__device__ __forceinline__ void dev_set_error(int32_t *err, int32_t code) {
    if (err) atomicCAS(err, 0, code);
}

// Index-checked build (compiled with -DNDFT_CHECKED into libndft_checked.so):
// the packing, fold, epilogue and direct-tile kernels test each computed
// global index against the extent their problem implies before the access; a
// failed test records kDevBadIndex in the plan's error word (ndft_query_error
// then returns NDFT_E_CUDA) and the access is skipped.  In the normal build the
// test compiles away.
#ifdef NDFT_CHECKED
__device__ __forceinline__ bool ndft_in(bool ok, int32_t *err) {
    if (!ok) dev_set_error(err, kDevBadIndex);
    return ok;
}
#else
__device__ __forceinline__ constexpr bool ndft_in(bool, int32_t *) { return true; }
#endif

// Event pair around the main contraction kernel of an exec call (no-ops unless
// ndft_timer_start armed the plan; recording an event allocates nothing).
inline void timer_begin(const Plan &p, cudaStream_t s) {
    if (p.tev && p.tcount < p.tcap) cudaEventRecord(p.tev[2 * p.tcount], s);
}
inline void timer_end(const Plan &p, cudaStream_t s) {
    if (p.tev && p.tcount < p.tcap) {
        cudaEventRecord(p.tev[2 * p.tcount + 1], s);
        ++p.tcount;
    }
}

// ---- launchers (defined in the .cu files) --------------------------------------

// tables.cu
cudaError_t launch_tables(int N, float2 *tw32, short2 *twq, cudaStream_t s);
cudaError_t tables_preload();  // loads the module of the table kernel (no launch)

// direct.cu
cudaError_t launch_direct_ndft(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s,
                               int *launches);
cudaError_t launch_direct_caf(const Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags,
                              void *A, cudaStream_t s, int *launches);
cudaError_t launch_direct_batched(const Plan &p, const void *surv, const void *ref, void *out,
                                  cudaStream_t s, int *launches);
size_t direct_ws_bytes(const ndft_desc &d, int sm_count);
cudaError_t direct_caf_preload();  // loads the fp32 CAF kernel's module and sets its attributes (no launch)
int direct_caf_splits(int N, int nlags, int nbins, int sm_count, int tune);

// nfft.cu
constexpr int64_t kNfftChunkBytes = 64ll << 20;  // intermediate per chunk: stays in the 129 MB L2
size_t nfft_ws_bytes(const ndft_desc &d, int64_t *chunk);
cudaError_t launch_nfft(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s, int *launches);
cudaError_t launch_nfft_bins(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s,
                             int *launches);
cudaError_t launch_nfft_caf(const Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags, void *A,
                            cudaStream_t s, int *launches);

// fft.cu
cudaError_t launch_fft_bins(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s,
                            int *launches);
cudaError_t launch_fft_caf(const Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags, void *A,
                           cudaStream_t s, int *launches);

// epilogue.cu
cudaError_t launch_reduce_splits(const float *ws, int nsplit, int64_t count, float *out, cudaStream_t s);
cudaError_t reduce_preload();  // loads the fp32 split-sum kernel's module (no launch)
// complex partials [nsplit][count] -> |sum| (fp32) per cell
cudaError_t launch_reduce_abs(const float2 *ws, int nsplit, int64_t count, float *out, cudaStream_t s);
cudaError_t launch_reduce_splits_i32(const uint32_t *ws, int nsplit, int64_t count, uint32_t *out,
                                     cudaStream_t s);
cudaError_t launch_argmax(const float2 *X, int64_t rows, int64_t cols, int64_t *idx, float *val,
                          cudaStream_t s);

// adjoint.cu
cudaError_t launch_caf_backward(const Plan &p, const void *s_ref, int lag0, int nlags, const void *dA,
                                void *ds, cudaStream_t s, int *launches);
cudaError_t launch_caf_backward_inputs(Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags,
                                       const void *dA, void *ds_surv, void *ds_ref, cudaStream_t s,
                                       int *launches);

// ternary.cu
bool ternary_supported(const ndft_desc &d);
size_t ternary_ws_bytes(const ndft_desc &d, int sm_count);
cudaError_t ternary_plan_init(Plan &p, cudaStream_t s);
cudaError_t launch_ternary_ndft(Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s,
                                int *launches);
cudaError_t launch_ternary_caf(Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags,
                               void *A, cudaStream_t s, int *launches);
cudaError_t ternary_batched_init(Plan &p, const ndft_cpi *cpis, int ncpi, cudaStream_t s);
cudaError_t launch_ternary_batched(Plan &p, const void *surv, const void *ref, void *out, cudaStream_t s,
                                   int *launches);
cudaError_t launch_ternary_adjoint(Plan &p, const void *s_ref, int lag0, int nlags, const void *dA, void *ds,
                                   cudaStream_t s, int *launches);
int ternary_adjoint_g_lags(const Plan &p, int nlags);
// G for nc lags: interleaved complex [nsplit][nc][N], or with *planar fp32
// [nsplit][2 nc][N] (Re of lag a in row 2 a, Im in 2 a + 1)
cudaError_t launch_ternary_adjoint_g(Plan &p, int nc, const void *dA, const float2 **G, int *nsplit,
                                     int64_t *split_stride, bool *planar, cudaStream_t s, int *launches);

}  // namespace ndft
