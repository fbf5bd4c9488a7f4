// adjoint.cu -- gradient of the nonlinear ambiguity surface (Eq. 12a) with
// respect to its inputs.
//
// Where no operand is 0, d(a (x) b)/da = sgn(b) and d(a (x) b)/db = sgn(a)
// (from Eq. 1-2).  Through Eq. 6 this makes z (x) W act on dz as
// multiplication by S = sigma(W) and s (x) c act on ds as multiplication by
// sigma(c) (on dc by sigma(s)), sigma(v) = sgn(v_r) + j sgn(v_i).  So, with
// dA = dL/dRe A + j dL/dIm A,
//     G_l[i]      = sum_k conj(S[p_k][i]) dA[l][k]       (transposed ternary contraction)
//     ds_surv[i]  = sum_l conj(sigma(c_l[i])) G_l[i],    c_l[i] = conj(s_ref[i - l])
//     ds_ref[j]   = sum_l conj(conj(sigma(s_surv[i])) G_l[i]),  i = j + l
// (without the conjugation of s_ref: no outer conj in ds_ref).
// k_caf_backward: one block owns 64 samples x 64 lags and walks the bins in
// chunks of 16; it either folds its lags into one ds_surv partial per sample
// (the partials of the lag tiles are summed in order by the split-K
// reduction) or stores G for k_grad_fold, which forms both gradients.
#include "internal.cuh"

#include <algorithm>

namespace ndft {

namespace {

constexpr int TI = 64, TL = 64, KB = 16;

__device__ __forceinline__ float sgnf(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

template <bool STORE_G>
__global__ void __launch_bounds__(256)
    k_caf_backward(const float2 *__restrict__ tw, const float2 *__restrict__ sref, int N, int p0, int nbins,
                   int lag0, int nlags, uint32_t flags, const float2 *__restrict__ dA, float2 *__restrict__ part) {
    __shared__ float2 sS[KB][TI + 1];   // conj(S[p][i]) as (sgn W_r, -sgn W_i)
    __shared__ float2 sD[KB][TL + 1];   // dA[l][p]
    __shared__ float2 red[16][TI + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.x * TI, l0 = blockIdx.y * TL;

    float2 acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[q][j] = make_float2(0.f, 0.f);

    // Staging: thread element r is (bin k0 + kk, sample i0 + c) with kk = e >> 6,
    // c = e & 63, e = tid + 256 r, the same sample for every k0; its twiddle
    // index m = ((p0 + k) i) mod N advances by (KB i) mod N per bin chunk.
    int64_t m[4], mstep[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = tid + 256 * r;
        const int kk = e >> 6, c = e & 63;
        const int64_t i = i0 + c;
        int64_t pm = ((int64_t)p0 + kk) % N;
        if (pm < 0) pm += N;
        m[r] = (pm * i) % N;
        mstep[r] = ((int64_t)KB * i) % N;
    }
    for (int k0 = 0; k0 < nbins; k0 += KB) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + 256 * r;
            const int kk = e >> 6, c = e & 63;
            // sign pattern for sample i0 + c at bin k0 + kk
            float2 sv = make_float2(0.f, 0.f);
            const int i = i0 + c, k = k0 + kk;
            if (i < N && k < nbins) {
                const float2 w = __ldg(&tw[m[r]]);
                sv = make_float2(sgnf(w.x), -sgnf(w.y));
            }
            m[r] += mstep[r];
            if (m[r] >= N) m[r] -= N;
            sS[kk][c] = sv;
            // upstream gradient for lag l0 + c at bin k0 + kk
            const int l = l0 + c;
            sD[kk][c] = (l < nlags && k < nbins) ? dA[(int64_t)l * nbins + k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KB; ++kk) {
            float2 s[4], d[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) s[j] = sS[kk][tx + 16 * j];  // samples tx + 16 j: no bank conflicts
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = sD[kk][ty * 4 + q];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // conj(S) * dA, conj(S) = (s.x, s.y) with s.y = -sgn(W_i)
                    acc[q][j].x += s[j].x * d[q].x - s[j].y * d[q].y;
                    acc[q][j].y += s[j].x * d[q].y + s[j].y * d[q].x;
                }
        }
        __syncthreads();
    }

    if constexpr (STORE_G) {
        // G[l][i] for this thread's 4 lags x 4 samples (part is [nlags][N])
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int l = l0 + ty * 4 + q;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = i0 + tx + 16 * j;
                if (l < nlags && i < N) part[(int64_t)l * N + i] = acc[q][j];
            }
        }
    } else {
    // multiply by conj(sigma(c_l[i])) and fold this thread's 4 lags
    float2 fold[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        fold[j] = make_float2(0.f, 0.f);
        const int i = i0 + tx + 16 * j;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int l = l0 + ty * 4 + q;
            if (i >= N || l >= nlags) continue;
            int64_t jj = (int64_t)i - ((int64_t)lag0 + l);
            if (flags & NDFT_F_CIRCULAR_LAG) {
                jj %= N;
                if (jj < 0) jj += N;
            }
            if (jj < 0 || jj >= N) continue;  // c = 0: no dependence
            const float2 r = sref[jj];
            const float cr = sgnf(r.x);
            const float ci = (flags & NDFT_F_NO_CONJ_REF) ? sgnf(r.y) : -sgnf(r.y);  // sigma(c)
            // conj(sigma(c)) * G = (cr - j ci)(g.x + j g.y)
            fold[j].x += cr * acc[q][j].x + ci * acc[q][j].y;
            fold[j].y += cr * acc[q][j].y - ci * acc[q][j].x;
        }
        red[ty][tx + 16 * j] = fold[j];
    }
    __syncthreads();
    if (tid < TI) {
        float2 t = make_float2(0.f, 0.f);
        for (int r = 0; r < 16; ++r) {
            t.x += red[r][tid].x;
            t.y += red[r][tid].y;
        }
        const int i = i0 + tid;
        if (i < N) part[(int64_t)blockIdx.y * N + i] = t;
    }
    }
}

// Both gradients from G ([nsplit][nc][N] complex, split partials summed here;
// with PLANAR fp32 [nsplit][2 nc][N], Re and Im of lag a in rows 2 a, 2 a + 1)
// for the nc lags lag_first .. lag_first + nc - 1.  A block owns 32
// consecutive indices t (one per lane) and warp w takes the lags w, w + 8, ...;
// the eight warp sums are added in warp order, so the result is deterministic.
// ds_surv[t] uses G at sample t, ds_ref[t] at sample t + l.  accumulate = 0
// stores, 1 adds to the previous chunk's values (in chunk order).
__device__ __forceinline__ float2 sigma2(float2 v) { return make_float2(sgnf(v.x), sgnf(v.y)); }

// G of lag a at sample i from split sp
template <bool PLANAR>
__device__ __forceinline__ float2 g_at(const float2 *__restrict__ G, int64_t split_stride, int N, int64_t a, int64_t i,
                                       int sp) {
    if constexpr (PLANAR) {
        const float *Gf = reinterpret_cast<const float *>(G) + 2 * sp * split_stride + 2 * a * N;
        return make_float2(Gf[i], Gf[N + i]);
    } else {
        return G[sp * split_stride + a * N + i];
    }
}

template <bool SURV, bool REF, bool PLANAR>
__global__ void __launch_bounds__(256)
    k_grad_fold(const float2 *__restrict__ G, int nsplit, int64_t split_stride, int N, int lag_first, int nc,
                uint32_t flags, const float2 *__restrict__ s_surv, const float2 *__restrict__ s_ref,
                float2 *__restrict__ ds_surv, float2 *__restrict__ ds_ref, int accumulate) {
    __shared__ float2 red[2][8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + lane;
    const bool circ = flags & NDFT_F_CIRCULAR_LAG, noconj = flags & NDFT_F_NO_CONJ_REF;
    float2 gs = make_float2(0.f, 0.f), gr = make_float2(0.f, 0.f);
    if (t < N) {
        // U lags at a time: every load of the group is issued before any of
        // its terms is formed (the kernel is bound by load latency); a pair
        // outside the signals reads index 0 and weighs its term by 0 (adding
        // an exact zero never changes these sums, which start at +0 and so
        // never hold -0)
        constexpr int U = 4;
        for (int a0 = w; a0 < nc; a0 += 8 * U) {
            float2 gsv[U], grv[U], rv[U], sv[U];
            bool ins[U], inr[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int a = a0 + 8 * u;
                const bool live = a < nc;
                const int ac = live ? a : w;
                const int64_t l = (int64_t)lag_first + ac;
                int64_t j = t - l, i = t + l;  // the s_ref / s_surv samples met at lag l
                if (circ) {
                    j %= N;
                    if (j < 0) j += N;
                    i %= N;
                    if (i < 0) i += N;
                }
                ins[u] = live && j >= 0 && j < N;
                inr[u] = live && i >= 0 && i < N;
                const int64_t ic = inr[u] ? i : 0;
                if (SURV) {
                    float2 g = g_at<PLANAR>(G, split_stride, N, ac, t, 0);
                    for (int sp = 1; sp < nsplit; ++sp) {
                        const float2 h = g_at<PLANAR>(G, split_stride, N, ac, t, sp);
                        g.x += h.x;
                        g.y += h.y;
                    }
                    gsv[u] = g;
                    rv[u] = __ldg(&s_ref[ins[u] ? j : 0]);
                }
                if (REF) {
                    float2 g = g_at<PLANAR>(G, split_stride, N, ac, ic, 0);
                    for (int sp = 1; sp < nsplit; ++sp) {
                        const float2 h = g_at<PLANAR>(G, split_stride, N, ac, ic, sp);
                        g.x += h.x;
                        g.y += h.y;
                    }
                    grv[u] = g;
                    sv[u] = __ldg(&s_surv[ic]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (SURV) {
                    const float2 g = gsv[u], r = rv[u];
                    const float cr = ins[u] ? sgnf(r.x) : 0.f;
                    const float ci = ins[u] ? (noconj ? sgnf(r.y) : -sgnf(r.y)) : 0.f;  // sigma(c)
                    gs.x += cr * g.x + ci * g.y;  // conj(sigma(c)) G
                    gs.y += cr * g.y - ci * g.x;
                }
                if (REF) {
                    const float2 g = grv[u];
                    const float2 sg = inr[u] ? sigma2(sv[u]) : make_float2(0.f, 0.f);
                    const float dr = sg.x * g.x + sg.y * g.y;  // conj(sigma(s)) G = dL/dc
                    const float di = sg.x * g.y - sg.y * g.x;
                    gr.x += dr;
                    gr.y += noconj ? di : -di;  // c = conj(s_ref): conjugate back
                }
            }
        }
    }
    red[0][w][lane] = gs;
    red[1][w][lane] = gr;
    __syncthreads();
    if (w < 2 && t < N) {
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v.x += red[w][k][lane].x;
            v.y += red[w][k][lane].y;
        }
        float2 *dst = w == 0 ? (SURV ? ds_surv : nullptr) : (REF ? ds_ref : nullptr);
        if (dst) {
            if (accumulate) {
                const float2 o = dst[t];
                v.x += o.x;
                v.y += o.y;
            }
            dst[t] = v;
        }
    }
}

}  // namespace

cudaError_t launch_caf_backward_inputs(Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags,
                                       const void *dA, void *ds_surv, void *ds_ref, cudaStream_t s,
                                       int *launches) {
    const int N = p.d.n, nb = p.d.nbins ? p.d.nbins : N;
    const float2 *dA2 = static_cast<const float2 *>(dA);
    // lags per pass: as many as the workspace holds G for
    bool tern = p.d.form == NDFT_FORM_TERNARY_GEMM;
    int chunk = tern ? ternary_adjoint_g_lags(p, nlags) : 0;
    if (chunk < 1) {
        tern = false;
        chunk = (int)std::min<int64_t>(nlags, (int64_t)(p.ws_alloc / ((size_t)N * sizeof(float2))));
    }
    if (chunk < 1) return cudaErrorNotSupported;
    cudaError_t e = cudaSuccess;
    for (int a0 = 0; a0 < nlags; a0 += chunk) {
        const int nc = std::min(chunk, nlags - a0);
        const float2 *G = nullptr;
        int nsplit = 1;
        int64_t sstride = 0;
        bool planar = false;
        if (tern) {
            if ((e = launch_ternary_adjoint_g(p, nc, dA2 + (int64_t)a0 * nb, &G, &nsplit, &sstride, &planar, s,
                                              launches)) != cudaSuccess)
                return e;
        } else {
            dim3 grid((N + TI - 1) / TI, (nc + TL - 1) / TL);
            timer_begin(p, s);
            k_caf_backward<true><<<grid, 256, 0, s>>>(p.tw32, nullptr, N, p.d.p0, nb, 0, nc, p.d.flags,
                                                      dA2 + (int64_t)a0 * nb, static_cast<float2 *>(p.ws));
            timer_end(p, s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            *launches += 1;
            G = static_cast<const float2 *>(p.ws);
        }
        const int blocks = (N + 31) / 32;
        auto *ss = static_cast<const float2 *>(s_surv);
        auto *sr = static_cast<const float2 *>(s_ref);
        auto *os = static_cast<float2 *>(ds_surv);
        auto *orf = static_cast<float2 *>(ds_ref);
        const int acc = a0 > 0;
        if (ds_surv && planar)
            k_grad_fold<true, true, true><<<blocks, 256, 0, s>>>(G, nsplit, sstride, N, lag0 + a0, nc, p.d.flags, ss,
                                                                 sr, os, orf, acc);
        else if (ds_surv)
            k_grad_fold<true, true, false><<<blocks, 256, 0, s>>>(G, nsplit, sstride, N, lag0 + a0, nc, p.d.flags, ss,
                                                                  sr, os, orf, acc);
        else if (planar)
            k_grad_fold<false, true, true><<<blocks, 256, 0, s>>>(G, nsplit, sstride, N, lag0 + a0, nc, p.d.flags, ss,
                                                                  sr, os, orf, acc);
        else
            k_grad_fold<false, true, false><<<blocks, 256, 0, s>>>(G, nsplit, sstride, N, lag0 + a0, nc, p.d.flags,
                                                                   ss, sr, os, orf, acc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 1;
    }
    return cudaSuccess;
}

cudaError_t launch_caf_backward(const Plan &p, const void *s_ref, int lag0, int nlags, const void *dA, void *ds,
                                cudaStream_t s, int *launches) {
    const int N = p.d.n, nb = p.d.nbins ? p.d.nbins : N;
    const int ltiles = (nlags + TL - 1) / TL;
    dim3 grid((N + TI - 1) / TI, ltiles);
    float2 *part = (ltiles == 1) ? static_cast<float2 *>(ds) : static_cast<float2 *>(p.ws);
    timer_begin(p, s);
    k_caf_backward<false><<<grid, 256, 0, s>>>(p.tw32, static_cast<const float2 *>(s_ref), N, p.d.p0, nb, lag0, nlags,
                                        p.d.flags, static_cast<const float2 *>(dA), part);
    timer_end(p, s);
    *launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || ltiles == 1) return e;
    *launches += 1;
    return launch_reduce_splits(reinterpret_cast<const float *>(part), ltiles, (int64_t)N * 2,
                                static_cast<float *>(ds), s);
}

}  // namespace ndft
