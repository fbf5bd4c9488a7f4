/*
 * ndft.h -- C ABI of the GB300 (sm_103a) library for the multiplication-free
 * nonlinear DFT of Bozkurt et al., arXiv 1402.0532.
 *
 * The operator (Eq. 1-2):  a (x) b = sgn(a b) (|a| + |b|), 0 if a or b is 0.
 * Complex extension (Eq. 6): a (x) b = a_r(x)b_r - a_i(x)b_i + j(a_i(x)b_r + b_i(x)a_r).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every data pointer is a DEVICE pointer (cudaMalloc'd or equivalent) owned
 *    by the caller, unless a parameter says "host".  The library never frees,
 *    keeps or reallocates caller memory.
 *  - complex64 data is interleaved float2 {re, im}, the layout of
 *    torch.complex64 / std::complex<float>.  Q1.14 data is interleaved int16
 *    pairs (value = q / 2^14) in, interleaved int32 pairs out.
 *  - Arrays are dense and row-major as stated per call; base pointers must be
 *    16-byte aligned, otherwise NDFT_E_INVALID.
 *  - Outputs must not overlap inputs or each other, except where a call says
 *    so (nfft_exec may run in place); calls reject outputs that start at an
 *    input's or another output's address with NDFT_E_INVALID.
 *  - Argument errors are returned synchronously and launch nothing.  CUDA
 *    launch errors are returned as NDFT_E_CUDA.  Errors detected inside a
 *    kernel (a bounded wait that ran out, an internal check) are recorded in
 *    the plan's device error word and returned by ndft_query_error().
 *  - Exec calls allocate nothing and never synchronise the stream; all
 *    memory they need is allocated by the plan.  One plan may serve one stream
 *    at a time.
 *  - Twiddles W^m = exp(-j 2 pi m / N) (defined under Eq. 8) are computed once
 *    per plan in fp64 from the angle reduced to a quadrant in integer
 *    arithmetic: values on the axes (m = 0, N/4, N/2, 3N/4) are exactly
 *    0 and +-1, and their signs are exact.
 */
#ifndef NDFT_H_
#define NDFT_H_

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NDFT_OK = 0,
    NDFT_E_INVALID = 1,      /* bad argument: null/misaligned pointer, size, combination */
    NDFT_E_UNSUPPORTED = 2,  /* valid request the library does not provide */
    NDFT_E_CUDA = 3,         /* a CUDA runtime call or launch failed */
    NDFT_E_NOMEM = 4,        /* device allocation at plan time failed */
    NDFT_E_TIMEOUT = 5,      /* a bounded device-side wait ran out (see ndft_query_error) */
    NDFT_E_OVERFLOW = 6      /* a Q1.14 sum left int32 (plans with NDFT_F_Q14_RANGE; see ndft_query_error) */
} ndft_status;

typedef enum {
    NDFT_FORM_DIRECT = 0,       /* (x) evaluated term by term on the CUDA cores */
    NDFT_FORM_TERNARY_GEMM = 1, /* a (x) b = sgn(b) a + sgn(a) b as two dense contractions on tcgen05 */
    NDFT_FORM_NFFT = 2,         /* the Sec. 3 NFFT in place of the NDFT (N a power of two <= 65536,
                                   FP32): ndft_exec gives the NFFT's bins p0 .. p0 + nbins - 1 and
                                   caf_exec Eq. 12a with the NFFT over each lag product */
    NDFT_FORM_FFT = 3           /* the ordinary DFT by a radix-2 FFT (N a power of two <= 65536,
                                   FP32): ndft_exec gives DFT bins, caf_exec Eq. 12b -- the lag
                                   product with (x), then the linear DFT */
} ndft_form;

typedef enum {
    NDFT_PREC_FP32 = 0,    /* complex64 in/out, fp32 arithmetic (DIRECT form, NFFT)          */
    NDFT_PREC_BF16X2 = 1,  /* complex64 in/out; bf16 hi+lo operands, exact ternary sign
                              matrices, fp32 accumulation (TERNARY_GEMM form)                */
    NDFT_PREC_Q14 = 2      /* int16 pairs (Q1.14) in, int32 pairs out; integer (x), sums
                              modulo 2^32 (DIRECT form)                                      */
} ndft_prec;

/* CAF options (Eq. 12a): the default conjugates s_ref and treats s_ref[j] as 0
 * outside [0, N) (linear correlation). */
#define NDFT_F_NO_CONJ_REF 0x1u  /* ablation: use s_ref[i-l] without the conjugate */
#define NDFT_F_CIRCULAR_LAG 0x2u /* index s_ref modulo N instead of zero padding    */
#define NDFT_F_NFFT_DIF 0x4u     /* NFFT by decimation in frequency (Sec. 3 names both
                                    FFT orders; the (x) butterflies make them differ):
                                    nfft_exec, and ndft_exec / caf_exec on NFFT plans */
#define NDFT_F_ABS_OUT 0x10u     /* caf_exec writes the magnitude surface |A| (fp32,
                                    [nlags][nbins]; |A| = sqrt(re^2 + im^2), each step
                                    rounded once) from the epilogue instead of A, on
                                    DIRECT fp32 and TERNARY_GEMM plans (single-CPI);
                                    ndft_exec returns NDFT_E_UNSUPPORTED on such plans */
#define NDFT_F_Q14_RANGE 0x8u    /* Q1.14 plans only: keep every output cell's sum exact
                                    (int64) besides the int32 result modulo 2^32, and
                                    report a cell whose sum left the int32 range through
                                    ndft_query_error (NDFT_E_OVERFLOW).  The output is
                                    the same either way; the sample axis of caf_exec
                                    is not split on such plans */

/* Plan descriptor.  Output bins are k = p0 .. p0 + nbins - 1 (signed, taken
 * modulo N); nbins = 0 means N bins starting at p0. */
typedef struct {
    int32_t n;          /* transform / CPI length N >= 1 (NFFT: power of two, 1..2^20) */
    int32_t p0;         /* first output bin */
    int32_t nbins;      /* number of output bins, 0 -> N */
    int32_t max_lags;   /* largest nlags a caf_exec / caf_backward call will pass (0: no CAF) */
    int64_t max_batch;  /* largest batch an ndft_exec / nfft_exec call will pass */
    int32_t form;       /* ndft_form */
    int32_t prec;       /* ndft_prec */
    uint32_t flags;     /* NDFT_F_* */
    int32_t reserved[3];/* must be 0 */
} ndft_desc;

typedef struct ndft_plan_s *ndft_plan_t;

/* One coherent processing interval (CPI) of a batched CAF: its s_surv / s_ref
 * start at element offsets off_surv / off_ref (complex elements, or int16
 * pairs for Q1.14) of the base pointers passed to caf_exec_batched, and its
 * surface A[nlags][nbins] at element offset off_out of the output base. */
typedef struct {
    int64_t off_surv, off_ref, off_out;
    int32_t n, lag0, nlags, p0, nbins;
    int32_t reserved;
} ndft_cpi;

/* ---- plan lifecycle ------------------------------------------------------ */

/* Creates a plan: validates d, allocates the twiddle tables (fp32; Q1.14 or the
 * ternary form's angle table), the workspace for max_batch / max_lags and the device
 * error word, and builds the tables on `stream` (fp64 on the GPU).
 * The ternary form accepts 1 <= N <= 2^18.  The plan
 * is ready once `stream` has reached this point.  Errors: NDFT_E_INVALID,
 * NDFT_E_UNSUPPORTED (form/prec pair not provided), NDFT_E_NOMEM, NDFT_E_CUDA. */
ndft_status ndft_plan(ndft_plan_t *out, const ndft_desc *d, cudaStream_t stream);

/* Creates a plan for caf_exec_batched over the `ncpi` CPIs listed in the HOST
 * array `cpis` (copied; the caller may free it on return).  form/prec/flags
 * as in ndft_desc.  The work list, per-CPI tables and workspace are built
 * here, once.  Each CPI: n >= 1, nlags >= 1, 1 <= nbins. */
ndft_status ndft_plan_batched(ndft_plan_t *out, const ndft_cpi *cpis, int32_t ncpi, int32_t form,
                              int32_t prec, uint32_t flags, cudaStream_t stream);

/* Releases everything the plan owns (synchronises the device first). */
ndft_status ndft_plan_destroy(ndft_plan_t plan);

/* ---- transforms ------------------------------------------------------------ */

/* NDFT, Eq. 8 (Sec. 2): X[b][k] = sum_n W^(((p0+k) n) mod N) (x) x[b][n].
 * x: [batch][N], X: [batch][nbins]; complex64 (FP32, BF16X2) or Q1.14.
 * 0 <= batch <= max_batch.  On an NDFT_FORM_NFFT plan: X[b][k] is bin
 * (p0 + k) mod N of the NFFT of x[b] (see nfft_exec), bit for bit; on an
 * NDFT_FORM_FFT plan the ordinary DFT bin (fp32 radix-2 FFT). */
ndft_status ndft_exec(ndft_plan_t plan, const void *x, void *X, int64_t batch, cudaStream_t stream);

/* NFFT, Sec. 3: radix-2 decimation in time with every twiddle product
 * replaced by (x) (also W^0 = 1); the 1-point NFFT is the identity; output
 * in natural order.  Per butterfly: t = W (x) O[k], X[k] = E[k] + t,
 * X[k + N/2] = E[k] - t, evaluated in fp32 in exactly that order, so results
 * are reproducible bit for bit.  Requires N a power of two, nbins = N, p0 = 0,
 * prec FP32.  x, X: [batch][N] complex64; X may equal x (in place).
 * With NDFT_F_NFFT_DIF (N <= 65536): decimation in frequency instead, natural
 * input, per butterfly on (E, O) = (x[n], x[n + L/2]) of a span-L block:
 * E' = E + O, O' = W_L^n (x) (E - O), recursing on both halves; natural-order
 * output (bin 2k from the first half, 2k + 1 from the second). */
ndft_status nfft_exec(ndft_plan_t plan, const void *x, void *X, int64_t batch, cudaStream_t stream);

/* Nonlinear cross-ambiguity surface, Eq. 12a (Sec. 4), read left to right:
 *   A[a][k] = sum_i ( s_surv[i] (x) conj(s_ref[i - l]) ) (x) W^((i p) mod N),
 *   l = lag0 + a (0 <= a < nlags), p = p0 + k (0 <= k < nbins),
 * s_ref[j] = 0 outside [0, N) unless NDFT_F_CIRCULAR_LAG.
 * s_surv, s_ref: [N]; A: [nlags][nbins]; 1 <= nlags <= max_lags and
 * lag0 + nlags - 1 <= INT32_MAX (NDFT_E_INVALID otherwise; the same bound holds
 * for caf_backward, caf_backward_inputs, caf_exec_noalloc and every batched CPI).
 * On an NDFT_FORM_NFFT plan the sum over i is the Sec. 3 NFFT of the lag
 * product z_l (computed in fp32 as above): A[a][k] = NFFT(z_l)[(p0 + k) mod N],
 * reproducible bit for bit.  On an NDFT_FORM_FFT plan it is the ordinary DFT
 * (Eq. 12b): A[a][k] = sum_i z_l[i] W^((i p) mod N), by an fp32 radix-2 FFT. */
ndft_status caf_exec(ndft_plan_t plan, const void *s_surv, const void *s_ref, int32_t lag0,
                     int32_t nlags, void *A, cudaStream_t stream);

/* Batched CAF over the plan's CPI list: CPI c reads surv_base + off_surv,
 * ref_base + off_ref and writes out_base + off_out.  Offsets are in elements
 * of the plan's precision.  The direct form runs one persistent launch over
 * all CPIs.  The tensor-core form, when every CPI's window pairs, runs one
 * conjugate-paired call per CPI (packing, contraction, fold; longest CPI
 * first, alternating between `stream` and a plan-owned side stream that
 * forks from and joins back into it, so capture in a CUDA graph works);
 * otherwise, or with tuning key 6 = 1, it packs every CPI and runs one
 * persistent unpaired contraction, which needs the whole batch's packed
 * operand (16 bytes per sample and lag of every CPI): a paired plan keeps
 * that only when it is at most 4 GiB, else key 6 = 1 gives
 * NDFT_E_UNSUPPORTED. */
ndft_status caf_exec_batched(ndft_plan_t plan, const void *surv_base, const void *ref_base,
                             void *out_base, cudaStream_t stream);

/* Adjoint of caf_exec with respect to s_surv (complex64 plans).  Given
 * dA = dL/dRe A + j dL/dIm A ([nlags][nbins]) returns
 *   ds[i] = dL/dRe s_surv[i] + j dL/dIm s_surv[i]
 *         = sum_l conj(sigma(c_l[i])) sum_p conj(S[p][i]) dA[l][p],
 * with c_l[i] = conj(s_ref[i-l]), S[p][i] = sigma(W^(i p)), sigma(v) =
 * sgn(v_r) + j sgn(v_i): the derivative d(a (x) b)/da = sgn(b) of Eq. 1-2
 * (valid where no operand is 0), chained through Eq. 6 and Eq. 12a.
 * ds: [N].  s_surv is not read (the derivative does not depend on it a.e.).
 * NDFT_E_UNSUPPORTED on Q1.14, NDFT_FORM_NFFT and NDFT_FORM_FFT plans. */
ndft_status caf_backward(ndft_plan_t plan, const void *s_surv, const void *s_ref, int32_t lag0,
                         int32_t nlags, const void *dA, void *ds, cudaStream_t stream);

/* Adjoint of caf_exec with respect to both inputs (complex64 plans).  With
 * G_l[i] = sum_p conj(S[p][i]) dA[l][p] as for caf_backward:
 *   ds_surv[i] = sum_l conj(sigma(c_l[i])) G_l[i]                  (= caf_backward)
 *   ds_ref[j]  = sum_l conj(conj(sigma(s_surv[i])) G_l[i]),  i = j + l
 * (i taken modulo N with NDFT_F_CIRCULAR_LAG, else only 0 <= i < N; with
 * NDFT_F_NO_CONJ_REF the outer conj is dropped): the derivative
 * d(a (x) b)/db = sgn(a) of Eq. 1-2 for the s_ref operand of the lag product,
 * chained through Eq. 6 and Eq. 12a.  ds_ref[j] = dL/dRe s_ref[j] + j dL/dIm
 * s_ref[j].  ds_surv may be NULL (then only ds_ref is formed); with ds_ref NULL
 * the call is caf_backward.  G is formed once for both, lag chunks as large as
 * the plan's workspace holds (the tensor cores on the ternary form, else CUDA
 * cores), then folded by a deterministic kernel.  s_surv, s_ref, ds_*: [N]
 * complex64; dA: [nlags][nbins] complex64; all device pointers, 16-byte
 * aligned (NDFT_E_INVALID otherwise).  NDFT_E_UNSUPPORTED on Q1.14,
 * NDFT_FORM_NFFT and NDFT_FORM_FFT plans. */
ndft_status caf_backward_inputs(ndft_plan_t plan, const void *s_surv, const void *s_ref, int32_t lag0,
                                int32_t nlags, const void *dA, void *ds_surv, void *ds_ref,
                                cudaStream_t stream);

/* Allocation-free variant of caf_exec for the direct fp32 form (the paper has
 * no counterpart: this serves callers that cannot allocate device memory at
 * the point of use, such as a real-time loop that forbids cudaMalloc after
 * start-up or code running during another thread's global-mode graph capture).
 * Same result as caf_exec on a direct fp32 plan with the same n, p0, nbins,
 * flags (up to fp32 summation order), with no plan: the twiddle table and the
 * split-K partials live in a 32 MiB static device array that every GPU loading
 * the library keeps until exit.  Limits: 1 <= n <= 2^20, 1 <= nbins <= n,
 * 1 <= nlags <= 2^20; beyond them NDFT_E_INVALID and nothing is launched.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and loads every kernel the call can launch; make it
 * before any stream capture.  After a reset of the device's context
 * (cudaDeviceReset) the next call repeats that set-up, so it too belongs
 * before any capture.  Calls share the array: calls that overlap on the GPU
 * race and must be serialised.
 * s_surv, s_ref: [n] complex64; A: [nlags][nbins] complex64; device pointers. */
ndft_status caf_exec_noalloc(int32_t n, int32_t p0, int32_t nbins, const void *s_surv, const void *s_ref,
                             int32_t lag0, int32_t nlags, uint32_t flags, void *A, cudaStream_t stream);

/* ---- epilogue helpers -------------------------------------------------------- */

/* Per row of X ([rows][cols] complex64): the index of the largest |X|^2
 * (re*re + im*im rounded in fp32), lowest index on ties -> idx[rows] (int64),
 * and that |X|^2 -> val[rows] (float, may be NULL).  The peak reading of
 * Eq. 9 / Fig. 1.  Needs no plan. */
ndft_status ndft_argmax(const void *X, int64_t rows, int64_t cols, int64_t *idx, float *val,
                        cudaStream_t stream);

/* ---- diagnostics ------------------------------------------------------------- */

/* Synchronises `stream`, returns the plan's device error word as a status
 * (NDFT_OK if none) and clears it: NDFT_E_TIMEOUT (a bounded wait ran out),
 * NDFT_E_OVERFLOW (a Q1.14 output cell's exact sum left int32, on plans with
 * NDFT_F_Q14_RANGE; the cell holds the sum modulo 2^32), NDFT_E_CUDA
 * (another device-side check).  The first error recorded since the last
 * query wins. */
ndft_status ndft_query_error(ndft_plan_t plan, cudaStream_t stream);

/* Copies one of the plan's tables to caller memory: which = 0 -> fp32
 * twiddles W^m, [N] float2; 1 -> Q1.14 twiddles, [N] int16 pairs (Q1.14
 * plans); 2 -> the ternary form's two-level angle table, [nth + 256] float2:
 * (cos, sin)((pi/2) 256 j / N) for j < nth = (N-1)/256 + 1, then
 * (cos, sin)((pi/2) j / N) for j < 256 (ternary plans).  Single-CPI plans. */
ndft_status ndft_get_twiddles(ndft_plan_t plan, int32_t which, void *dst, cudaStream_t stream);

/* Bytes of device memory the plan holds (tables + workspace). */
ndft_status ndft_plan_bytes(ndft_plan_t plan, int64_t *bytes);

/* Kernel-launch count of the plan's last exec call (for accounting). */
ndft_status ndft_last_launches(ndft_plan_t plan, int32_t *count);

/* Tile / split choice for the plan's kernels: key 0 = split count along the
 * sample axis (0 = automatic); key 1 = ternary-GEMM tile (256: 256 rows in one
 * CTA with one tensor-memory accumulator pair; 128: 128 rows with two
 * accumulators used in turn; 258: the 256-row tile on a 2-SM pair, M = 256
 * MMAs with each CTA holding half of A and of B and two tensor-memory
 * accumulators used in turn, so that one chain's fold-out runs under the next
 * chain's MMAs; 0, the default: the 2-SM pair for the conjugate-paired
 * contraction with its A operand from the plan's table (key 7 = 0), 256
 * everywhere else); key 2 = ternary-GEMM K blocks
 * per tensor-memory accumulation chain before it is folded into the fp32
 * result (0 = the default: 64 blocks of 8 samples, or of 16 samples in the
 * conjugate-paired contraction of key 6); key 3 = ternary-GEMM fold path (0: bulk
 * tensor stores/adds, 1: per-element adds).  Used by the autotuner; affects
 * speed and fp32 rounding only.  Key 4 (test only) = 1: the ternary GEMM's
 * operand loader issues no loads, so every bounded wait of the kernel runs out
 * (about 2 s): the kernel abandons its work, releases its tensor memory and
 * returns, the output is left unspecified and ndft_query_error reports
 * NDFT_E_TIMEOUT; the plan stays usable once the key is set back to 0.
 * Key 5 = ternary-GEMM column parts of a single exec call: 1 (default) = one
 * part; 0 runs calls of at least 512 columns (lags, or NDFT vectors) as two
 * parts, the first of half the columns rounded down to a multiple of 256, so
 * that the second part's packing runs on a plan-owned side stream under the
 * first part's contraction (the side stream forks from and joins back into the
 * call's stream, so stream order and CUDA-graph capture are unaffected); a
 * multiple of 256 = two parts, the first of that many columns.  Two parts
 * shorten short bursts of calls by about 1 % but lengthen long runs at the
 * power limit by about 3 % (measured on the 65536-sample, 1024 x 1024 surface).
 * Key 6 = ternary-GEMM conjugate pairing: 0 (default) contracts bins +c and -c
 * together wherever that takes fewer tensor-core steps (W^(-c i) =
 * conj(W^(c i)), Eq. 8, so both bins come from one pair of real contractions
 * U = S_r v + F_r sigma(v), V = S_i v + F_i sigma(v): X[+c] = U + jV,
 * X[-c] = U - jV, half the multiply-adds per bin; bin 0 is summed by the
 * packing kernel); 1 = never; 2 = wherever the window allows it.  Pairing is
 * used with 256-row tiles (key 1 = 0, 256, or 258 with the A table) and one
 * column part only.  Same bar, different fp32 rounding.
 * Key 7 = the paired contraction's A operand (the S/F rows of Eq. 6 for
 * frequencies 1 .. S in bf16 hi/lo): 0 (default) = loaded by TMA from a table
 * the plan builds at creation (16 MiB per 1024 samples of a 1024-bin window;
 * built only while it stays within 2 GiB), 1 = generated on chip per K block
 * by producer warps from the twiddle table (the only form for larger tables).
 * Same bar either way.
 * Key 8 = the paired contraction's B operand (the lag products, or NDFT
 * inputs, as bf16 hi/lo and signs) on the 2-SM pair tile: 0 (default) or 3 =
 * packed just in time by the tile's own warps into the plan's workspace: each
 * CTA packs the 16-block x 64-column items of its own future loads that no
 * other CTA has claimed, at most key 9 items (default 4) ahead of its loads,
 * and loads an item once it is marked packed (bounded waits, NDFT_E_TIMEOUT
 * past them); 1 = packed by a separate kernel before the contraction; 2 =
 * formed in shared memory per K block by every tile that uses it (four times
 * per B tile; slower, for measurement).  The operand is the same in all
 * three, so every bin but bin 0 (whose sum is grouped differently) is the
 * same bit for bit.
 * Key 9 = items the key 8 = 0/3 packers may run ahead of their CTA's loads
 * (0 = 4).  Key 10 = the paired adjoint's A operand (the sign rows
 * sigma(W^(c i)), one row per sample, K over frequencies), which CAF plans
 * build as a table at creation (kblocks x 128-byte rows per 256 samples,
 * 277 MB for 65536 samples and 513 frequencies; within 2 GiB): 0 (default) =
 * from the table for caf_backward's contraction and generated on chip for
 * caf_backward_inputs' (there the table measured 2 % slower), 2 = from the
 * table for both, 1 = generated for both.  The same bits in every case. */
ndft_status ndft_set_tuning(ndft_plan_t plan, int32_t key, int32_t value);

/* Read-only facts about a plan and its last exec call, into *value:
 * key 0 = S, the largest frequency min(p, N - p) of the bin window (ternary
 *         plans; the paired contraction has rows for frequencies 1 .. S);
 * key 1 = the contraction variant of the last exec call: 0 none or not a
 *         tensor-core call, 1 one row pair per bin, 2 conjugate-paired rows;
 * key 2 = the sample-axis split count of the last exec call's contraction
 *         (0 if none);
 * key 3 = the tile of that contraction: 256 or 128 rows on one CTA, 258 the
 *         256-row tile on a 2-SM pair (0 if none).
 * NDFT_E_INVALID for another key or a NULL argument. */
ndft_status ndft_plan_query(ndft_plan_t plan, int32_t key, int64_t *value);

/* Device timing of the plan's main contraction kernel (the tensor-core GEMM,
 * the direct tile kernel, the NFFT or the adjoint kernel).  ndft_timer_start
 * creates `capacity` CUDA event pairs (0 disarms and frees them); every later
 * exec call then records one pair on its stream immediately around that kernel,
 * until capacity pairs are used.  ndft_timer_read synchronises on the recorded
 * events, returns the summed elapsed milliseconds and the number of timed
 * launches, and rearms the pairs.  Exec calls stay allocation-free. */
ndft_status ndft_timer_start(ndft_plan_t plan, int32_t capacity);
ndft_status ndft_timer_read(ndft_plan_t plan, double *ms_total, int32_t *count);

const char *ndft_status_string(ndft_status s);

/* Library version as an integer (major * 10000 + minor * 100 + patch). */
int32_t ndft_version(void);

/* Text of the last CUDA error behind an NDFT_E_CUDA / NDFT_E_NOMEM status
 * returned on the calling host thread ("no error" if none); static storage. */
const char *ndft_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NDFT_H_ */
