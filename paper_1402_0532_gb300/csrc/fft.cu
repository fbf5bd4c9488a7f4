// fft.cu -- the ordinary (linear) DFT by a radix-2 FFT in fp32, for Eq. 12b:
// the cross-ambiguity surface whose lag product is formed with the operator of
// Eq. 6 and whose sum over samples is the usual DFT, and for binned DFT output
// of a vector (ndft_exec on an NDFT_FORM_FFT plan).  Same kernels as the
// nonlinear FFT (fft_core.cuh) with the complex product in the butterfly, in
// decimation-in-frequency order (natural-order reads of the lag product; any
// order gives the linear DFT up to rounding).
#include "fft_core.cuh"

namespace ndft {

cudaError_t launch_fft_bins(const Plan &p, const void *x, void *X, int64_t batch, cudaStream_t s,
                            int *launches) {
    return fft_bins<OpLin, true>(p, x, X, batch, s, launches);
}

cudaError_t launch_fft_caf(const Plan &p, const void *s_surv, const void *s_ref, int lag0, int nlags, void *A,
                           cudaStream_t s, int *launches) {
    return fft_caf<OpLin, true>(p, s_surv, s_ref, lag0, nlags, A, s, launches);
}

}  // namespace ndft
