// adjoint.cu -- gradient of the nonlinear ambiguity surface (Eq. 12a) with
// respect to the surveillance signal.
//
// Where no operand is 0, d(a (x) b)/da = sgn(b) (from Eq. 1-2).  Through Eq. 6
// this makes z (x) W act on dz as multiplication by S = sigma(W) and s (x) c
// act on ds as multiplication by sigma(c), sigma(v) = sgn(v_r) + j sgn(v_i).
// So, with dA = dL/dRe A + j dL/dIm A,
//     G_l[i] = sum_k conj(S[p_k][i]) dA[l][k]            (transposed ternary contraction)
//     ds[i]  = sum_l conj(sigma(c_l[i])) G_l[i],  c_l[i] = conj(s_ref[i - l]).
// One block owns 64 samples x 64 lags, walks the bins in chunks of 16, then
// folds its lags into one partial per sample; the partials of the lag tiles
// are summed in order by the split-K reduction.
#include "internal.cuh"

namespace ndft {

namespace {

constexpr int TI = 64, TL = 64, KB = 16;

__device__ __forceinline__ float sgnf(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

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
            int64_t jj = (int64_t)i - (lag0 + l);
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

}  // namespace

cudaError_t launch_caf_backward(const Plan &p, const void *s_ref, int lag0, int nlags, const void *dA, void *ds,
                                cudaStream_t s, int *launches) {
    const int N = p.d.n, nb = p.d.nbins ? p.d.nbins : N;
    const int ltiles = (nlags + TL - 1) / TL;
    dim3 grid((N + TI - 1) / TI, ltiles);
    float2 *part = (ltiles == 1) ? static_cast<float2 *>(ds) : static_cast<float2 *>(p.ws);
    timer_begin(p, s);
    k_caf_backward<<<grid, 256, 0, s>>>(p.tw32, static_cast<const float2 *>(s_ref), N, p.d.p0, nb, lag0, nlags,
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
