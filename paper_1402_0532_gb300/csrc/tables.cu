// tables.cu -- per-plan twiddle tables, built once on the GPU in fp64.
//
// W^m = exp(-j 2 pi m / N) (W is defined under Eq. 8 of the paper).  The angle
// 2 pi m / N is split in integers as q (pi/2) + a with q = floor(4m / N),
// r = 4m - qN and a = (pi/2) r / N, so the axis values (r = 0) are exactly
// 0 / +-1 and every sign is exact.  This kernel is the only fp64 use on the GPU.
#include "internal.cuh"

namespace ndft {

__global__ void k_tables(int N, float2 *__restrict__ tw32, short2 *__restrict__ twq) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double half_pi = 1.5707963267948966;
    if (m < N) {
        const int64_t u = 4 * m;
        const int64_t q = u / N;
        const int64_t r = u - q * N;
        const double a = half_pi * ((double)r / (double)N);
        const double c = cos(a), s = sin(a);
        double ct, st;
        switch (q) {
            case 0: ct = c; st = s; break;
            case 1: ct = -s; st = c; break;
            case 2: ct = -c; st = -s; break;
            default: ct = s; st = -c; break;
        }
        const double wr = ct + 0.0, wi = -st + 0.0;  // +0 on the axes
        if (tw32) tw32[m] = make_float2(__double2float_rn(wr), __double2float_rn(wi));
        if (twq) twq[m] = make_short2((short)rint(wr * 16384.0), (short)rint(wi * 16384.0));
    }
}

cudaError_t tables_preload() {
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, k_tables);
}

cudaError_t launch_tables(int N, float2 *tw32, short2 *twq, cudaStream_t s) {
    const int64_t count = N;
    const int threads = 256;
    const int blocks = (int)((count + threads - 1) / threads);
    k_tables<<<blocks, threads, 0, s>>>(N, tw32, twq);
    return cudaGetLastError();
}

}  // namespace ndft
