// epilogue.cu -- split-K reduction and peak search.
//
// Split-K: partial surfaces [nsplit][count] are summed in split order, so the
// result does not depend on scheduling.  fp32 sums round as written; the
// Q1.14 partials are added modulo 2^32 (associative, hence exact).
// Peak search: the largest |X|^2 per row, lowest index on ties (the peak
// reading of Eq. 9 / Fig. 1).
#include "internal.cuh"

namespace ndft {

namespace {

__global__ void k_reduce_f32(const float *__restrict__ ws, int nsplit, int64_t count, float *__restrict__ out) {
    const int64_t n4 = (count % 4 == 0) ? count / 4 : 0;  // float4 rows stay 16-byte aligned
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 a = reinterpret_cast<const float4 *>(ws)[i];
        for (int s = 1; s < nsplit; ++s) {
            const float4 b = reinterpret_cast<const float4 *>(ws + (int64_t)s * count)[i];
            a.x = __fadd_rn(a.x, b.x);
            a.y = __fadd_rn(a.y, b.y);
            a.z = __fadd_rn(a.z, b.z);
            a.w = __fadd_rn(a.w, b.w);
        }
        reinterpret_cast<float4 *>(out)[i] = a;
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        float a = ws[i];
        for (int s = 1; s < nsplit; ++s) a = __fadd_rn(a, ws[(int64_t)s * count + i]);
        out[i] = a;
    }
}

// Split-K sum of complex partials [nsplit][count] (float2), in split order,
// then the magnitude sqrt(re^2 + im^2) with each operation rounded once.
__global__ void k_reduce_abs(const float2 *__restrict__ ws, int nsplit, int64_t count, float *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        float2 a = ws[i];
        for (int s = 1; s < nsplit; ++s) {
            const float2 b = ws[(int64_t)s * count + i];
            a.x = __fadd_rn(a.x, b.x);
            a.y = __fadd_rn(a.y, b.y);
        }
        out[i] = __fsqrt_rn(__fadd_rn(__fmul_rn(a.x, a.x), __fmul_rn(a.y, a.y)));
    }
}

__global__ void k_reduce_u32(const uint32_t *__restrict__ ws, int nsplit, int64_t count, uint32_t *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        uint32_t a = 0;
        for (int s = 0; s < nsplit; ++s) a += ws[(int64_t)s * count + i];
        out[i] = a;
    }
}

__device__ __forceinline__ void better(float &v, int64_t &i, float v2, int64_t i2) {
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

__global__ void k_argmax(const float2 *__restrict__ X, int64_t cols, int64_t *__restrict__ idx,
                         float *__restrict__ val) {
    const int64_t row = blockIdx.x;
    const float2 *x = X + row * cols;
    float bv = -1.0f;
    int64_t bi = INT64_MAX;
    for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) {
        const float2 v = x[c];
        const float m = __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y));
        better(bv, bi, m, c);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const int64_t i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        better(bv, bi, v2, i2);
    }
    __shared__ float sv[32];
    __shared__ int64_t si[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sv[w] = bv;
        si[w] = bi;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        bv = l < nw ? sv[l] : -1.0f;
        bi = l < nw ? si[l] : INT64_MAX;
        for (int o = 16; o > 0; o >>= 1) {
            const float v2 = __shfl_xor_sync(0xffffffffu, bv, o);
            const int64_t i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            better(bv, bi, v2, i2);
        }
        if (l == 0) {
            idx[row] = bi;
            if (val) val[row] = bv;
        }
    }
}

int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t reduce_preload() {
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, k_reduce_f32);
}

cudaError_t launch_reduce_splits(const float *ws, int nsplit, int64_t count, float *out, cudaStream_t s) {
    k_reduce_f32<<<grid_for(count / 4 + 1, 256), 256, 0, s>>>(ws, nsplit, count, out);
    return cudaGetLastError();
}

cudaError_t launch_reduce_abs(const float2 *ws, int nsplit, int64_t count, float *out, cudaStream_t s) {
    k_reduce_abs<<<grid_for(count, 256), 256, 0, s>>>(ws, nsplit, count, out);
    return cudaGetLastError();
}

cudaError_t launch_reduce_splits_i32(const uint32_t *ws, int nsplit, int64_t count, uint32_t *out,
                                     cudaStream_t s) {
    k_reduce_u32<<<grid_for(count, 256), 256, 0, s>>>(ws, nsplit, count, out);
    return cudaGetLastError();
}

cudaError_t launch_argmax(const float2 *X, int64_t rows, int64_t cols, int64_t *idx, float *val,
                          cudaStream_t s) {
    if (rows == 0) return cudaSuccess;
    if (rows > 0x7fffffff) return cudaErrorInvalidValue;
    const int threads = cols >= 4096 ? 1024 : (cols >= 256 ? 256 : 32);
    k_argmax<<<(unsigned)rows, threads, 0, s>>>(X, cols, idx, val);
    return cudaGetLastError();
}

}  // namespace ndft
