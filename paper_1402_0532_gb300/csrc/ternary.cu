// ternary.cu -- placeholder until the tensor-core form lands.
#include "internal.cuh"

namespace ndft {
bool ternary_supported(const ndft_desc &) { return false; }
size_t ternary_ws_bytes(const ndft_desc &, int) { return 0; }
cudaError_t ternary_plan_init(Plan &, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_ternary_ndft(Plan &, const void *, void *, int64_t, cudaStream_t, int *) {
    return cudaErrorNotSupported;
}
cudaError_t launch_ternary_caf(Plan &, const void *, const void *, int, int, void *, cudaStream_t, int *) {
    return cudaErrorNotSupported;
}
}  // namespace ndft
