/*
 * ndft_oracle.c -- slow, literal CPU oracle for the nonlinear DFT (NDFT),
 * the nonlinear FFT (NFFT) and the nonlinear cross-ambiguity function of
 * Bozkurt et al., "Approximate Computation of DFT without Performing Any
 * Multiplications: Applications to Radar Signal Processing" (arXiv 1402.0532).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU library
 * shares no code, header, table or constant generator with this file.
 *
 * Everything here evaluates the operator the way the paper defines it:
 *   - real a (x) b by the three sign cases of Eq. 2 and |a|+|b| of Eq. 1,
 *   - complex a (x) b by the four real terms of Eq. 6,
 *   - sums in plain left-to-right order in double precision.
 * The identity a (x) b = sgn(b) a + sgn(a) b is deliberately NOT used here;
 * the tests use it only as an independent cross-check.
 *
 * Readings of points the paper leaves open:
 *   twiddles  W^m = exp(-j 2 pi m / N) with the angle reduced to a quadrant
 *             in integer arithmetic, so values on the axes are exact
 *             (cos = 0 exactly at m = N/4, 3N/4; sin = 0 at m = 0, N/2).
 *   NDFT      X[k] = sum_n W^((k n) mod N) (x) x[n]           (Eq. 8, Sec. 2)
 *   NFFT      radix-2 decimation in time, every twiddle product replaced by
 *             (x), including W^0; output in natural order      (Sec. 3)
 *   CAF       A[l,p] = sum_i (s_surv[i] (x) conj(s_ref[i-l])) (x) W^(i p)
 *             left-associative, s_ref conjugated, s_ref[j] = 0 outside
 *             [0, N)                                           (Eq. 12a, Sec. 4)
 *   Q1.14     integer inputs, integer (x), exact 64-bit sums reduced
 *             modulo 2^32 (two's complement wrap).
 *   adjoint   d(a (x) b)/da = sgn(b) for a != 0 (derivative of Eq. 1-2),
 *             chained through Eq. 6 and Eq. 12a.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_F_NO_CONJ_REF 0x1u  /* ablation: s_ref not conjugated       */
#define ORACLE_F_CIRCULAR_LAG 0x2u /* s_ref index taken modulo N           */

/* ------------------------------------------------------------------------ */
/* Eq. 1 and Eq. 2: the real additive operator.                              */
/* ------------------------------------------------------------------------ */
static int sign_of_product(double a, double b) {
    /* Eq. 2: +1 when a, b share a sign, -1 when they differ, 0 otherwise. */
    if ((a > 0 && b > 0) || (a < 0 && b < 0)) return 1;
    if ((a < 0 && b > 0) || (a > 0 && b < 0)) return -1;
    return 0;
}

double oracle_otimes(double a, double b) {
    int s = sign_of_product(a, b);
    if (s == 0) return 0.0;                 /* "otherwise" case: exactly +0 */
    double m = fabs(a) + fabs(b);           /* Eq. 1 */
    return s > 0 ? m : -m;
}

static float otimes_f32(float a, float b) {
    int s;
    if ((a > 0 && b > 0) || (a < 0 && b < 0)) s = 1;
    else if ((a < 0 && b > 0) || (a > 0 && b < 0)) s = -1;
    else return 0.0f;
    float m = fabsf(a) + fabsf(b);          /* one fp32 rounding */
    return s > 0 ? m : -m;
}

static int64_t otimes_i64(int64_t a, int64_t b) {
    int s;
    if ((a > 0 && b > 0) || (a < 0 && b < 0)) s = 1;
    else if ((a < 0 && b > 0) || (a > 0 && b < 0)) s = -1;
    else return 0;
    int64_t m = (a < 0 ? -a : a) + (b < 0 ? -b : b);
    return s > 0 ? m : -m;
}

/* Eq. 6: a (x) b = a_r(x)b_r - a_i(x)b_i + j (a_i(x)b_r + b_i(x)a_r). */
static void cot64(double ar, double ai, double br, double bi, double *cr, double *ci) {
    double t1 = oracle_otimes(ar, br);
    double t2 = oracle_otimes(ai, bi);
    double t3 = oracle_otimes(ai, br);
    double t4 = oracle_otimes(bi, ar);
    *cr = t1 - t2;
    *ci = t3 + t4;
}

static void cot32(float ar, float ai, float br, float bi, float *cr, float *ci) {
    float t1 = otimes_f32(ar, br);
    float t2 = otimes_f32(ai, bi);
    float t3 = otimes_f32(ai, br);
    float t4 = otimes_f32(bi, ar);
    *cr = t1 - t2;
    *ci = t3 + t4;
}

static void cot_i64(int64_t ar, int64_t ai, int64_t br, int64_t bi, int64_t *cr, int64_t *ci) {
    *cr = otimes_i64(ar, br) - otimes_i64(ai, bi);
    *ci = otimes_i64(ai, br) + otimes_i64(bi, ar);
}

void oracle_cotimes(const double *a, const double *b, double *out) {
    cot64(a[0], a[1], b[0], b[1], &out[0], &out[1]);
}

/* Eq. 3: <x (.) y> = sum_i x_i (x) y_i, summed in index order. */
double oracle_vecprod(const double *x, const double *y, int64_t n) {
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) acc += oracle_otimes(x[i], y[i]);
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Twiddles W^m = exp(-j 2 pi m / N)   (W is defined under Eq. 8).          */
/* The angle 2 pi m / N is split as q (pi/2) + a with q = floor(4m/N) and   */
/* a = (pi/2) r / N, r = 4m - qN, all in integers; a = 0 gives cos = 1 and  */
/* sin = 0 exactly, so the axis values are exact.                          */
/* ------------------------------------------------------------------------ */
static int64_t mod_pos(int64_t a, int64_t n) {
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

void oracle_twiddle(int64_t N, int64_t m, double *out) {
    m = mod_pos(m, N);
    int64_t u = 4 * m;
    int64_t q = u / N;
    int64_t r = u - q * N;
    double a = 1.5707963267948966 * ((double)r / (double)N);
    double c = cos(a), s = sin(a);
    double ct, st; /* cos(theta), sin(theta) */
    switch (q) {
        case 0: ct = c;  st = s;  break;
        case 1: ct = -s; st = c;  break;
        case 2: ct = -c; st = -s; break;
        default: ct = s; st = -c; break;
    }
    out[0] = ct + 0.0;   /* +0.0 instead of -0.0 on the axes */
    out[1] = -st + 0.0;
}

/* Q1.14 twiddle: round-half-even of 2^14 W^m; the axis zeros stay exact. */
void oracle_twiddle_q14(int64_t N, int64_t m, int32_t *out) {
    double w[2];
    oracle_twiddle(N, m, w);
    out[0] = (int32_t)nearbyint(w[0] * 16384.0);
    out[1] = (int32_t)nearbyint(w[1] * 16384.0);
}

/* Q1.14 copy of the whole table (int16 pairs). */
void oracle_twiddle_table_q14(int64_t N, int16_t *out) {
    for (int64_t m = 0; m < N; ++m) {
        int32_t w[2];
        oracle_twiddle_q14(N, m, w);
        out[2 * m] = (int16_t)w[0];
        out[2 * m + 1] = (int16_t)w[1];
    }
}

static double *twiddle_table64(int64_t N) {
    double *t = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    if (!t) return NULL;
    for (int64_t m = 0; m < N; ++m) oracle_twiddle(N, m, t + 2 * m);
    return t;
}

/* fp32 copy of the same twiddles: each component rounded once from fp64. */
void oracle_twiddle_table_f32(int64_t N, float *out) {
    for (int64_t m = 0; m < N; ++m) {
        double w[2];
        oracle_twiddle(N, m, w);
        out[2 * m] = (float)w[0];
        out[2 * m + 1] = (float)w[1];
    }
}

/* ------------------------------------------------------------------------ */
/* NDFT, Eq. 8: X[k] = sum_n W^((k n) mod N) (x) x[n].                       */
/* Bins k = p0 .. p0+nbins-1 (signed, taken mod N).                          */
/* x: [batch][N] complex interleaved, X: [batch][nbins] complex interleaved. */
/* ------------------------------------------------------------------------ */
int oracle_ndft(const double *x, int64_t batch, int64_t N, int64_t p0, int64_t nbins, double *X) {
    if (N <= 0 || batch < 0 || nbins < 0) return 1;
    double *W = twiddle_table64(N);
    if (!W) return 2;
#pragma omp parallel for schedule(dynamic)
    for (int64_t cell = 0; cell < batch * nbins; ++cell) {
        int64_t b = cell / nbins, k = cell % nbins;
        int64_t p = mod_pos(p0 + k, N);
        const double *xb = x + 2 * b * N;
        double re = 0.0, im = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            int64_t m = (p * n) % N;
            double cr, ci;
            cot64(W[2 * m], W[2 * m + 1], xb[2 * n], xb[2 * n + 1], &cr, &ci);
            re += cr;
            im += ci;
        }
        X[2 * cell] = re;
        X[2 * cell + 1] = im;
    }
    free(W);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* NFFT, Sec. 3: the radix-2 decimation-in-time recursion with every         */
/* twiddle product replaced by (x).  N-point NFFT of x:                      */
/*   E = NFFT(x[0::2]), O = NFFT(x[1::2])  (N/2 points each)                 */
/*   t = W_N^k (x) O[k];  X[k] = E[k] + t;  X[k + N/2] = E[k] - t            */
/* and the 1-point NFFT is the identity.  W_N^k = W_Nfull^(k Nfull / N).     */
/* ------------------------------------------------------------------------ */
static void nfft_rec64(const double *x, int64_t n, int64_t stride, const double *W, int64_t Nfull,
                       double *out, double *scratch) {
    if (n == 1) {
        out[0] = x[0];
        out[1] = x[1];
        return;
    }
    int64_t h = n / 2;
    double *E = scratch, *O = scratch + 2 * h, *sub = scratch + 2 * n;
    nfft_rec64(x, h, 2 * stride, W, Nfull, E, sub);
    nfft_rec64(x + 2 * stride, h, 2 * stride, W, Nfull, O, sub);
    int64_t step = Nfull / n;
    for (int64_t k = 0; k < h; ++k) {
        double tr, ti;
        cot64(W[2 * k * step], W[2 * k * step + 1], O[2 * k], O[2 * k + 1], &tr, &ti);
        out[2 * k] = E[2 * k] + tr;
        out[2 * k + 1] = E[2 * k + 1] + ti;
        out[2 * (k + h)] = E[2 * k] - tr;
        out[2 * (k + h) + 1] = E[2 * k + 1] - ti;
    }
}

static void nfft_rec32(const float *x, int64_t n, int64_t stride, const float *W, int64_t Nfull,
                       float *out, float *scratch) {
    if (n == 1) {
        out[0] = x[0];
        out[1] = x[1];
        return;
    }
    int64_t h = n / 2;
    float *E = scratch, *O = scratch + 2 * h, *sub = scratch + 2 * n;
    nfft_rec32(x, h, 2 * stride, W, Nfull, E, sub);
    nfft_rec32(x + 2 * stride, h, 2 * stride, W, Nfull, O, sub);
    int64_t step = Nfull / n;
    for (int64_t k = 0; k < h; ++k) {
        float tr, ti;
        cot32(W[2 * k * step], W[2 * k * step + 1], O[2 * k], O[2 * k + 1], &tr, &ti);
        out[2 * k] = E[2 * k] + tr;
        out[2 * k + 1] = E[2 * k + 1] + ti;
        out[2 * (k + h)] = E[2 * k] - tr;
        out[2 * (k + h) + 1] = E[2 * k + 1] - ti;
    }
}

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

int oracle_nfft(const double *x, int64_t batch, int64_t N, double *X) {
    if (!is_pow2(N) || batch < 0) return 1;
    double *W = twiddle_table64(N);
    if (!W) return 2;
    int err = 0;
#pragma omp parallel
    {
        /* scratch: 2 complex per level, bounded by 4N complex in total */
        double *scr = (double *)malloc(sizeof(double) * 8 * (size_t)N + 64);
        if (!scr) {
#pragma omp atomic write
            err = 2;
        } else {
#pragma omp for schedule(dynamic)
            for (int64_t b = 0; b < batch; ++b)
                nfft_rec64(x + 2 * b * N, N, 1, W, N, X + 2 * b * N, scr);
            free(scr);
        }
    }
    free(W);
    return err;
}

/* The same recursion evaluated in fp32 arithmetic (one rounding per real    */
/* (x), per subtraction/addition), with the fp32-rounded twiddles.           */
int oracle_nfft_f32(const float *x, int64_t batch, int64_t N, float *X) {
    if (!is_pow2(N) || batch < 0) return 1;
    float *W = (float *)malloc(sizeof(float) * 2 * (size_t)N);
    if (!W) return 2;
    oracle_twiddle_table_f32(N, W);
    int err = 0;
#pragma omp parallel
    {
        float *scr = (float *)malloc(sizeof(float) * 8 * (size_t)N + 64);
        if (!scr) {
#pragma omp atomic write
            err = 2;
        } else {
#pragma omp for schedule(dynamic)
            for (int64_t b = 0; b < batch; ++b)
                nfft_rec32(x + 2 * b * N, N, 1, W, N, X + 2 * b * N, scr);
            free(scr);
        }
    }
    free(W);
    return err;
}

/* ------------------------------------------------------------------------ */
/* NFFT by decimation in frequency (Sec. 3 names both FFT orders; with (x)   */
/* in the butterflies the two give different transforms).  N-point DIF of x: */
/*   Y[m] = x[m] + x[m + N/2],  Z[m] = W_N^m (x) (x[m] - x[m + N/2]),        */
/*   m < N/2;  X[2k] = DIF(Y)[k],  X[2k + 1] = DIF(Z)[k];                    */
/* the 1-point transform is the identity.                                    */
/* ------------------------------------------------------------------------ */
static void nfft_dif_rec64(const double *x, int64_t n, const double *W, int64_t Nfull, double *out,
                           double *scratch) {
    if (n == 1) {
        out[0] = x[0];
        out[1] = x[1];
        return;
    }
    int64_t h = n / 2, step = Nfull / n;
    double *Y = scratch, *Z = scratch + 2 * h, *YY = scratch + 2 * n, *ZZ = YY + 2 * h, *sub = scratch + 4 * n;
    for (int64_t m = 0; m < h; ++m) {
        double ar = x[2 * m], ai = x[2 * m + 1], br = x[2 * (m + h)], bi = x[2 * (m + h) + 1];
        Y[2 * m] = ar + br;
        Y[2 * m + 1] = ai + bi;
        cot64(W[2 * m * step], W[2 * m * step + 1], ar - br, ai - bi, &Z[2 * m], &Z[2 * m + 1]);
    }
    nfft_dif_rec64(Y, h, W, Nfull, YY, sub);
    nfft_dif_rec64(Z, h, W, Nfull, ZZ, sub);
    for (int64_t k = 0; k < h; ++k) {
        out[4 * k] = YY[2 * k];
        out[4 * k + 1] = YY[2 * k + 1];
        out[4 * k + 2] = ZZ[2 * k];
        out[4 * k + 3] = ZZ[2 * k + 1];
    }
}

static void nfft_dif_rec32(const float *x, int64_t n, const float *W, int64_t Nfull, float *out, float *scratch) {
    if (n == 1) {
        out[0] = x[0];
        out[1] = x[1];
        return;
    }
    int64_t h = n / 2, step = Nfull / n;
    float *Y = scratch, *Z = scratch + 2 * h, *YY = scratch + 2 * n, *ZZ = YY + 2 * h, *sub = scratch + 4 * n;
    for (int64_t m = 0; m < h; ++m) {
        float ar = x[2 * m], ai = x[2 * m + 1], br = x[2 * (m + h)], bi = x[2 * (m + h) + 1];
        Y[2 * m] = ar + br;
        Y[2 * m + 1] = ai + bi;
        float dr = ar - br, di = ai - bi;
        cot32(W[2 * m * step], W[2 * m * step + 1], dr, di, &Z[2 * m], &Z[2 * m + 1]);
    }
    nfft_dif_rec32(Y, h, W, Nfull, YY, sub);
    nfft_dif_rec32(Z, h, W, Nfull, ZZ, sub);
    for (int64_t k = 0; k < h; ++k) {
        out[4 * k] = YY[2 * k];
        out[4 * k + 1] = YY[2 * k + 1];
        out[4 * k + 2] = ZZ[2 * k];
        out[4 * k + 3] = ZZ[2 * k + 1];
    }
}

int oracle_nfft_dif(const double *x, int64_t batch, int64_t N, double *X) {
    if (!is_pow2(N) || batch < 0) return 1;
    double *W = twiddle_table64(N);
    if (!W) return 2;
    int err = 0;
#pragma omp parallel
    {
        double *scr = (double *)malloc(sizeof(double) * 8 * (size_t)N + 64);
        if (!scr) {
#pragma omp atomic write
            err = 2;
        } else {
#pragma omp for schedule(dynamic)
            for (int64_t b = 0; b < batch; ++b)
                nfft_dif_rec64(x + 2 * b * N, N, W, N, X + 2 * b * N, scr);
            free(scr);
        }
    }
    free(W);
    return err;
}

int oracle_nfft_dif_f32(const float *x, int64_t batch, int64_t N, float *X) {
    if (!is_pow2(N) || batch < 0) return 1;
    float *W = (float *)malloc(sizeof(float) * 2 * (size_t)N);
    if (!W) return 2;
    oracle_twiddle_table_f32(N, W);
    int err = 0;
#pragma omp parallel
    {
        float *scr = (float *)malloc(sizeof(float) * 8 * (size_t)N + 64);
        if (!scr) {
#pragma omp atomic write
            err = 2;
        } else {
#pragma omp for schedule(dynamic)
            for (int64_t b = 0; b < batch; ++b)
                nfft_dif_rec32(x + 2 * b * N, N, W, N, X + 2 * b * N, scr);
            free(scr);
        }
    }
    free(W);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Conditioning of the NFFT (Sec. 3, either order) in fp32.  (x) jumps where */
/* an operand crosses zero, so an fp32 evaluation of the recursion stays     */
/* close to the fp64 one only while every data operand of every (x) keeps    */
/* its fp64 sign.  This evaluates the fp64 recursion (the same values as     */
/* oracle_nfft / oracle_nfft_dif) and beside each value a bound on how far   */
/* an fp32 evaluation of it (fp32 twiddles, one rounding per (x) and per     */
/* addition) can be from it, by running error analysis: with u = 2^-24,      */
/*   input (fp32 data)                     e = 0                            */
/*   twiddle component w                   e = u |w|                        */
/*   real a (x) b, both signs kept         e = (e_a + e_b)(1 + u) + u' |r|   */
/*   c = a +- b                            e = (e_a + e_b)(1 + u) + u' |c|   */
/* (u' = u + 2^-52 also covers the rounding of the fp64 value itself).  A    */
/* data operand v keeps its sign in fp32 if |v| > e_v, or v = 0 with e_v = 0;*/
/* stable[b] = 1 if that holds for every (x) of vector b, and then           */
/* |X32 - X64| <= bound elementwise (per component).                         */
/* ------------------------------------------------------------------------ */
#define U32 5.9604644775390625e-08 /* 2^-24 */
#define U32P (5.9604644775390625e-08 + 2.220446049250313e-16)

static int keeps_sign(double v, double e) { return fabs(v) > e || (v == 0.0 && e == 0.0); }

/* real (x) with the twiddle component w (sign exact in fp32) and the data
 * operand v: value and bound; clears *ok when v may change sign */
static double ox_bound(double w, double v, double ev, double *e, int *ok) {
    if (!keeps_sign(v, ev)) *ok = 0;
    double r = oracle_otimes(w, v);
    /* an exact zero on either side gives exactly 0 in fp32 as well */
    *e = (w == 0.0 || (v == 0.0 && ev == 0.0)) ? 0.0 : (U32 * fabs(w) + ev) * (1.0 + U32) + U32P * fabs(r);
    return r;
}

/* complex W (x) v with bounds, Eq. 6 in the operand order of cot64 */
static void cot_bound(double wr, double wi, double vr, double vi, double evr, double evi, double *cr,
                      double *ci, double *ecr, double *eci, int *ok) {
    double e1, e2, e3, e4;
    double t1 = ox_bound(wr, vr, evr, &e1, ok);
    double t2 = ox_bound(wi, vi, evi, &e2, ok);
    double t3 = ox_bound(wi, vr, evr, &e3, ok);
    double t4 = ox_bound(wr, vi, evi, &e4, ok); /* vi (x) wr: (x) commutes exactly */
    *cr = t1 - t2;
    *ci = t3 + t4;
    *ecr = (e1 + e2) * (1.0 + U32) + U32P * fabs(*cr);
    *eci = (e3 + e4) * (1.0 + U32) + U32P * fabs(*ci);
}

static double add_bound(double c, double ea, double eb) { return (ea + eb) * (1.0 + U32) + U32P * fabs(c); }

/* values v[2n] and bounds e[2n] (Re, Im interleaved in both) */
static void nfft_bnd_dit(const double *x, const double *ex, int64_t n, int64_t stride, const double *W,
                         int64_t Nfull, double *out, double *eout, double *scr, int *ok) {
    if (n == 1) {
        out[0] = x[0];
        out[1] = x[1];
        eout[0] = ex[0];
        eout[1] = ex[1];
        return;
    }
    int64_t h = n / 2;
    double *E = scr, *O = scr + 2 * h, *eE = scr + 2 * n, *eO = eE + 2 * h, *sub = scr + 4 * n;
    nfft_bnd_dit(x, ex, h, 2 * stride, W, Nfull, E, eE, sub, ok);
    nfft_bnd_dit(x + 2 * stride, ex + 2 * stride, h, 2 * stride, W, Nfull, O, eO, sub, ok);
    int64_t step = Nfull / n;
    for (int64_t k = 0; k < h; ++k) {
        double tr, ti, etr, eti;
        cot_bound(W[2 * k * step], W[2 * k * step + 1], O[2 * k], O[2 * k + 1], eO[2 * k], eO[2 * k + 1], &tr,
                  &ti, &etr, &eti, ok);
        out[2 * k] = E[2 * k] + tr;
        out[2 * k + 1] = E[2 * k + 1] + ti;
        out[2 * (k + h)] = E[2 * k] - tr;
        out[2 * (k + h) + 1] = E[2 * k + 1] - ti;
        eout[2 * k] = add_bound(out[2 * k], eE[2 * k], etr);
        eout[2 * k + 1] = add_bound(out[2 * k + 1], eE[2 * k + 1], eti);
        eout[2 * (k + h)] = add_bound(out[2 * (k + h)], eE[2 * k], etr);
        eout[2 * (k + h) + 1] = add_bound(out[2 * (k + h) + 1], eE[2 * k + 1], eti);
    }
}

static void nfft_bnd_dif(const double *x, const double *ex, int64_t n, const double *W, int64_t Nfull,
                         double *out, double *eout, double *scr, int *ok) {
    if (n == 1) {
        out[0] = x[0];
        out[1] = x[1];
        eout[0] = ex[0];
        eout[1] = ex[1];
        return;
    }
    int64_t h = n / 2, step = Nfull / n;
    double *Y = scr, *Z = scr + 2 * h, *YY = scr + 2 * n, *ZZ = YY + 2 * h;
    double *eY = scr + 4 * n, *eZ = eY + 2 * h, *eYY = scr + 6 * n, *eZZ = eYY + 2 * h, *sub = scr + 8 * n;
    for (int64_t m = 0; m < h; ++m) {
        double ar = x[2 * m], ai = x[2 * m + 1], br = x[2 * (m + h)], bi = x[2 * (m + h) + 1];
        Y[2 * m] = ar + br;
        Y[2 * m + 1] = ai + bi;
        eY[2 * m] = add_bound(Y[2 * m], ex[2 * m], ex[2 * (m + h)]);
        eY[2 * m + 1] = add_bound(Y[2 * m + 1], ex[2 * m + 1], ex[2 * (m + h) + 1]);
        double dr = ar - br, di = ai - bi;
        double edr = add_bound(dr, ex[2 * m], ex[2 * (m + h)]);
        double edi = add_bound(di, ex[2 * m + 1], ex[2 * (m + h) + 1]);
        cot_bound(W[2 * m * step], W[2 * m * step + 1], dr, di, edr, edi, &Z[2 * m], &Z[2 * m + 1], &eZ[2 * m],
                  &eZ[2 * m + 1], ok);
    }
    nfft_bnd_dif(Y, eY, h, W, Nfull, YY, eYY, sub, ok);
    nfft_bnd_dif(Z, eZ, h, W, Nfull, ZZ, eZZ, sub, ok);
    for (int64_t k = 0; k < h; ++k) {
        out[4 * k] = YY[2 * k];
        out[4 * k + 1] = YY[2 * k + 1];
        out[4 * k + 2] = ZZ[2 * k];
        out[4 * k + 3] = ZZ[2 * k + 1];
        eout[4 * k] = eYY[2 * k];
        eout[4 * k + 1] = eYY[2 * k + 1];
        eout[4 * k + 2] = eZZ[2 * k];
        eout[4 * k + 3] = eZZ[2 * k + 1];
    }
}

/* x: [batch][N] complex (values representable in fp32); X and bound: [batch][N]
 * complex-interleaved; stable: [batch] */
int oracle_nfft_bound(const double *x, int64_t batch, int64_t N, int dif, double *X, double *bound,
                      int32_t *stable) {
    if (!is_pow2(N) || batch < 0) return 1;
    double *W = twiddle_table64(N);
    if (!W) return 2;
    int err = 0;
#pragma omp parallel
    {
        double *scr = (double *)malloc(sizeof(double) * (20 * (size_t)N + 64));
        double *ex = (double *)calloc(2 * (size_t)N, sizeof(double));
        if (!scr || !ex) {
#pragma omp atomic write
            err = 2;
        } else {
#pragma omp for schedule(dynamic)
            for (int64_t b = 0; b < batch; ++b) {
                int ok = 1;
                if (dif)
                    nfft_bnd_dif(x + 2 * b * N, ex, N, W, N, X + 2 * b * N, bound + 2 * b * N, scr, &ok);
                else
                    nfft_bnd_dit(x + 2 * b * N, ex, N, 1, W, N, X + 2 * b * N, bound + 2 * b * N, scr, &ok);
                stable[b] = ok;
            }
        }
        free(scr);
        free(ex);
    }
    free(W);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Lag product of Eq. 12a: z_l[i] = s_surv[i] (x) conj(s_ref[i - l]).        */
/* ------------------------------------------------------------------------ */
static int64_t ref_index(int64_t i, int64_t l, int64_t N, uint32_t flags) {
    int64_t j = i - l;
    if (flags & ORACLE_F_CIRCULAR_LAG) return mod_pos(j, N);
    return (j < 0 || j >= N) ? -1 : j;
}

static void lagprod64(const double *ss, const double *sr, int64_t N, int64_t l, uint32_t flags,
                      int64_t i, double *zr, double *zi) {
    int64_t j = ref_index(i, l, N, flags);
    double rr = 0.0, ri = 0.0;
    if (j >= 0) {
        rr = sr[2 * j];
        ri = (flags & ORACLE_F_NO_CONJ_REF) ? sr[2 * j + 1] : -sr[2 * j + 1];
    }
    cot64(ss[2 * i], ss[2 * i + 1], rr, ri, zr, zi);
}

int oracle_lagprod(const double *s_surv, const double *s_ref, int64_t N, int64_t lag, uint32_t flags,
                   double *z) {
    for (int64_t i = 0; i < N; ++i) lagprod64(s_surv, s_ref, N, lag, flags, i, &z[2 * i], &z[2 * i + 1]);
    return 0;
}

int oracle_lagprod_f32(const float *s_surv, const float *s_ref, int64_t N, int64_t lag, uint32_t flags,
                       float *z) {
    for (int64_t i = 0; i < N; ++i) {
        int64_t j = ref_index(i, lag, N, flags);
        float rr = 0.0f, ri = 0.0f;
        if (j >= 0) {
            rr = s_ref[2 * j];
            ri = (flags & ORACLE_F_NO_CONJ_REF) ? s_ref[2 * j + 1] : -s_ref[2 * j + 1];
        }
        cot32(s_surv[2 * i], s_surv[2 * i + 1], rr, ri, &z[2 * i], &z[2 * i + 1]);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* CAF, Eq. 12a (left-associative): A[l,p] = sum_i z_l[i] (x) W^((i p) mod N) */
/* for lags l = lag0 .. lag0+nlags-1 and bins p = p0 .. p0+nbins-1.          */
/* A: [nlags][nbins] complex interleaved.                                     */
/* If z32 != 0 the lag products are formed in fp32 from fp32 copies of the   */
/* signals (the element-wise stage in the GPU's precision) and the rest in    */
/* fp64; otherwise everything is fp64.                                        */
/* ------------------------------------------------------------------------ */
static int caf_cells(const double *s_surv, const double *s_ref, int64_t N, const int64_t *lags,
                     const int64_t *bins, int64_t ncells, uint32_t flags, int z32, double *A) {
    double *W = twiddle_table64(N);
    if (!W) return 2;
    float *ss32 = NULL, *sr32 = NULL;
    if (z32) {
        ss32 = (float *)malloc(sizeof(float) * 2 * (size_t)N);
        sr32 = (float *)malloc(sizeof(float) * 2 * (size_t)N);
        if (!ss32 || !sr32) { free(W); free(ss32); free(sr32); return 2; }
        for (int64_t i = 0; i < 2 * N; ++i) { ss32[i] = (float)s_surv[i]; sr32[i] = (float)s_ref[i]; }
    }
#pragma omp parallel for schedule(dynamic)
    for (int64_t c = 0; c < ncells; ++c) {
        int64_t l = lags[c], p = mod_pos(bins[c], N);
        double re = 0.0, im = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double zr, zi;
            if (z32) {
                int64_t j = ref_index(i, l, N, flags);
                float rr = 0.0f, ri = 0.0f, fr, fi;
                if (j >= 0) {
                    rr = sr32[2 * j];
                    ri = (flags & ORACLE_F_NO_CONJ_REF) ? sr32[2 * j + 1] : -sr32[2 * j + 1];
                }
                cot32(ss32[2 * i], ss32[2 * i + 1], rr, ri, &fr, &fi);
                zr = fr;
                zi = fi;
            } else {
                lagprod64(s_surv, s_ref, N, l, flags, i, &zr, &zi);
            }
            int64_t m = (i * p) % N;
            double cr, ci;
            cot64(zr, zi, W[2 * m], W[2 * m + 1], &cr, &ci);
            re += cr;
            im += ci;
        }
        A[2 * c] = re;
        A[2 * c + 1] = im;
    }
    free(W);
    free(ss32);
    free(sr32);
    return 0;
}

int oracle_caf(const double *s_surv, const double *s_ref, int64_t N, int64_t lag0, int64_t nlags,
               int64_t p0, int64_t nbins, uint32_t flags, int z32, double *A) {
    if (N <= 0 || nlags < 0 || nbins < 0) return 1;
    int64_t nc = nlags * nbins;
    int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc + 1));
    int64_t *P = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc + 1));
    if (!L || !P) { free(L); free(P); return 2; }
    for (int64_t c = 0; c < nc; ++c) { L[c] = lag0 + c / nbins; P[c] = p0 + c % nbins; }
    int rc = caf_cells(s_surv, s_ref, N, L, P, nc, flags, z32, A);
    free(L);
    free(P);
    return rc;
}

/* Selected cells only: (lags[c], bins[c]) for c < ncells -> A[c]. */
int oracle_caf_cells(const double *s_surv, const double *s_ref, int64_t N, const int64_t *lags,
                     const int64_t *bins, int64_t ncells, uint32_t flags, int z32, double *A) {
    if (N <= 0 || ncells < 0) return 1;
    return caf_cells(s_surv, s_ref, N, lags, bins, ncells, flags, z32, A);
}

/* ------------------------------------------------------------------------ */
/* Q1.14 fixed point.  Inputs int16 pairs (value = q / 2^14), twiddles       */
/* round(2^14 W).  (x) on integers is scale-consistent: (c a)(x)(c b) =      */
/* c (a (x) b) for c > 0, so integer results are 2^14 x the real ones.       */
/* Sums are exact in 64 bits and returned modulo 2^32 (two's complement).    */
/* The return value is 0, or 16 + (number of results whose exact sum does   */
/* not fit in int32) capped, so callers can see that wrap happened.          */
/* ------------------------------------------------------------------------ */
static int32_t wrap32(int64_t v) { return (int32_t)(uint32_t)(uint64_t)v; }

int oracle_ndft_q14(const int16_t *x, int64_t batch, int64_t N, int64_t p0, int64_t nbins, int32_t *X,
                    int64_t *n_overflow) {
    if (N <= 0 || batch < 0 || nbins < 0) return 1;
    int32_t *W = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)N);
    if (!W) return 2;
    for (int64_t m = 0; m < N; ++m) oracle_twiddle_q14(N, m, W + 2 * m);
    int64_t novf = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : novf)
    for (int64_t cell = 0; cell < batch * nbins; ++cell) {
        int64_t b = cell / nbins, k = cell % nbins;
        int64_t p = mod_pos(p0 + k, N);
        const int16_t *xb = x + 2 * b * N;
        int64_t re = 0, im = 0;
        for (int64_t n = 0; n < N; ++n) {
            int64_t m = (p * n) % N, cr, ci;
            cot_i64(W[2 * m], W[2 * m + 1], xb[2 * n], xb[2 * n + 1], &cr, &ci);
            re += cr;
            im += ci;
        }
        if (re != (int64_t)wrap32(re) || im != (int64_t)wrap32(im)) novf += 1;
        X[2 * cell] = wrap32(re);
        X[2 * cell + 1] = wrap32(im);
    }
    free(W);
    if (n_overflow) *n_overflow = novf;
    return 0;
}

int oracle_caf_q14(const int16_t *s_surv, const int16_t *s_ref, int64_t N, int64_t lag0, int64_t nlags,
                   int64_t p0, int64_t nbins, uint32_t flags, int32_t *A, int64_t *n_overflow) {
    if (N <= 0 || nlags < 0 || nbins < 0) return 1;
    int32_t *W = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)N);
    if (!W) return 2;
    for (int64_t m = 0; m < N; ++m) oracle_twiddle_q14(N, m, W + 2 * m);
    int64_t novf = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : novf)
    for (int64_t cell = 0; cell < nlags * nbins; ++cell) {
        int64_t l = lag0 + cell / nbins, p = mod_pos(p0 + cell % nbins, N);
        int64_t re = 0, im = 0;
        for (int64_t i = 0; i < N; ++i) {
            int64_t j = ref_index(i, l, N, flags);
            int64_t rr = 0, ri = 0, zr, zi, cr, ci;
            if (j >= 0) {
                rr = s_ref[2 * j];
                ri = (flags & ORACLE_F_NO_CONJ_REF) ? s_ref[2 * j + 1] : -(int64_t)s_ref[2 * j + 1];
            }
            cot_i64(s_surv[2 * i], s_surv[2 * i + 1], rr, ri, &zr, &zi);
            int64_t m = (i * p) % N;
            cot_i64(zr, zi, W[2 * m], W[2 * m + 1], &cr, &ci);
            re += cr;
            im += ci;
        }
        if (re != (int64_t)wrap32(re) || im != (int64_t)wrap32(im)) novf += 1;
        A[2 * cell] = wrap32(re);
        A[2 * cell + 1] = wrap32(im);
    }
    free(W);
    if (n_overflow) *n_overflow = novf;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the CAF with respect to s_surv, chained through the real      */
/* partial derivatives of Eq. 1-2: d(a (x) b)/da = sgn(b) where a != 0.      */
/* With G_A = dL/dRe A + j dL/dIm A given per cell, returns                  */
/* ds[i] = dL/dRe s_surv[i] + j dL/dIm s_surv[i].                            */
/*  stage 2 (z (x) W):  dRe/dz_r = sgn(W_r), dRe/dz_i = -sgn(W_i),          */
/*                      dIm/dz_r = sgn(W_i), dIm/dz_i =  sgn(W_r)           */
/*  stage 1 (s (x) c):  dz_r/ds_r = sgn(c_r), dz_r/ds_i = -sgn(c_i),        */
/*                      dz_i/ds_r = sgn(c_i), dz_i/ds_i =  sgn(c_r)         */
/* (each read off Eq. 6 with d(a (x) b)/da = sgn(b)).                        */
/* ------------------------------------------------------------------------ */
static double sgn(double v) { return v > 0 ? 1.0 : (v < 0 ? -1.0 : 0.0); }

/* dL/dz_r, dL/dz_i of z_l[i] (l = lag0 + a): the stage-2 partials summed over */
/* the bins of lag a. */
static void adj_gz(const double *W, int64_t N, int64_t i, int64_t a, int64_t p0, int64_t nbins,
                   const double *dA, double *gzr, double *gzi) {
    double r = 0.0, q = 0.0;
    for (int64_t k = 0; k < nbins; ++k) {
        int64_t p = mod_pos(p0 + k, N);
        int64_t m = (i * p) % N;
        double swr = sgn(W[2 * m]), swi = sgn(W[2 * m + 1]);
        double ar = dA[2 * (a * nbins + k)], ai = dA[2 * (a * nbins + k) + 1];
        r += ar * swr + ai * swi;
        q += ar * (-swi) + ai * swr;
    }
    *gzr = r;
    *gzi = q;
}

/* ds[i] (with respect to s_surv) */
static void adj_surv_at(const double *s_ref, const double *W, int64_t N, int64_t lag0, int64_t nlags, int64_t p0,
                        int64_t nbins, uint32_t flags, const double *dA, int64_t i, double *out) {
    double gr = 0.0, gi = 0.0;
    for (int64_t a = 0; a < nlags; ++a) {
        int64_t l = lag0 + a;
        int64_t j = ref_index(i, l, N, flags);
        double cr = 0.0, ci = 0.0;
        if (j >= 0) {
            cr = s_ref[2 * j];
            ci = (flags & ORACLE_F_NO_CONJ_REF) ? s_ref[2 * j + 1] : -s_ref[2 * j + 1];
        }
        double gzr, gzi;
        adj_gz(W, N, i, a, p0, nbins, dA, &gzr, &gzi);
        double scr = sgn(cr), sci = sgn(ci);
        gr += gzr * scr + gzi * sci;
        gi += gzr * (-sci) + gzi * scr;
    }
    out[0] = gr;
    out[1] = gi;
}

int oracle_caf_adjoint(const double *s_surv, const double *s_ref, int64_t N, int64_t lag0, int64_t nlags,
                       int64_t p0, int64_t nbins, uint32_t flags, const double *dA, double *ds) {
    if (N <= 0 || nlags < 0 || nbins < 0) return 1;
    double *W = twiddle_table64(N);
    if (!W) return 2;
    (void)s_surv;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) adj_surv_at(s_ref, W, N, lag0, nlags, p0, nbins, flags, dA, i, ds + 2 * i);
    free(W);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the CAF with respect to s_ref, by the same chain rule with the */
/* other operand of the lag product: d(a (x) b)/db = sgn(a) where b != 0.    */
/*  stage 1 (s (x) c):  dz_r/dc_r = sgn(s_r), dz_r/dc_i = -sgn(s_i),        */
/*                      dz_i/dc_r = sgn(s_i), dz_i/dc_i =  sgn(s_r)         */
/*  and c = conj(s_ref[j]) (s_ref[j] with the no-conjugate flag) negates    */
/*  the imaginary component.  For each j the lags l that read s_ref[j] are  */
/*  those with ref_index(i, l) = j, i.e. i = j + l (modulo N when the lag   */
/*  is circular; otherwise only 0 <= i < N).                                */
/* dref[j] = dL/dRe s_ref[j] + j dL/dIm s_ref[j].                            */
/* ------------------------------------------------------------------------ */
/* dref[j] (with respect to s_ref) */
static void adj_ref_at(const double *s_surv, const double *W, int64_t N, int64_t lag0, int64_t nlags, int64_t p0,
                       int64_t nbins, uint32_t flags, const double *dA, int64_t j, double *out) {
    double gr = 0.0, gi = 0.0;
    for (int64_t a = 0; a < nlags; ++a) {
        int64_t l = lag0 + a;
        int64_t i = j + l;
        if (flags & ORACLE_F_CIRCULAR_LAG) i = mod_pos(i, N);
        else if (i < 0 || i >= N) continue; /* no sample reads s_ref[j] at this lag */
        double gzr, gzi;
        adj_gz(W, N, i, a, p0, nbins, dA, &gzr, &gzi);
        double ssr = sgn(s_surv[2 * i]), ssi = sgn(s_surv[2 * i + 1]);
        double gcr = gzr * ssr + gzi * ssi;    /* dL/dc_r */
        double gci = gzr * (-ssi) + gzi * ssr; /* dL/dc_i */
        gr += gcr;
        gi += (flags & ORACLE_F_NO_CONJ_REF) ? gci : -gci;
    }
    out[0] = gr;
    out[1] = gi;
}

int oracle_caf_adjoint_ref(const double *s_surv, const double *s_ref, int64_t N, int64_t lag0, int64_t nlags,
                           int64_t p0, int64_t nbins, uint32_t flags, const double *dA, double *dref) {
    if (N <= 0 || nlags < 0 || nbins < 0) return 1;
    double *W = twiddle_table64(N);
    if (!W) return 2;
    (void)s_ref;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < N; ++j) adj_ref_at(s_surv, W, N, lag0, nlags, p0, nbins, flags, dA, j, dref + 2 * j);
    free(W);
    return 0;
}

/* Either adjoint at listed indices only (which = 0: s_surv, 1: s_ref), for */
/* sampled checks of large transforms. */
int oracle_caf_adjoint_at(const double *s_surv, const double *s_ref, int64_t N, int64_t lag0, int64_t nlags,
                          int64_t p0, int64_t nbins, uint32_t flags, const double *dA, int32_t which,
                          const int64_t *idx, int64_t nidx, double *out) {
    if (N <= 0 || nlags < 0 || nbins < 0 || nidx < 0 || (which != 0 && which != 1)) return 1;
    for (int64_t e = 0; e < nidx; ++e)
        if (idx[e] < 0 || idx[e] >= N) return 1;
    double *W = twiddle_table64(N);
    if (!W) return 2;
#pragma omp parallel for schedule(dynamic)
    for (int64_t e = 0; e < nidx; ++e) {
        if (which == 0) adj_surv_at(s_ref, W, N, lag0, nlags, p0, nbins, flags, dA, idx[e], out + 2 * e);
        else adj_ref_at(s_surv, W, N, lag0, nlags, p0, nbins, flags, dA, idx[e], out + 2 * e);
    }
    free(W);
    return 0;
}

/* Threads the OpenMP runtime will use (reported by the CPU baseline). */
#ifdef _OPENMP
#include <omp.h>
int oracle_num_threads(void) { return omp_get_max_threads(); }
#else
int oracle_num_threads(void) { return 1; }
#endif
