// noalloc.cu -- caf_exec_noalloc: the direct-form nonlinear CAF for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a surface:
// a real-time processing loop whose policy forbids device allocation after
// start-up (cudaMalloc can synchronise the device and its latency is
// unbounded), code that runs while another thread captures a CUDA graph in
// global mode (cudaMalloc is illegal then), or a host whose device memory is
// entirely reserved by an allocator it does not own.  A plan allocates its
// tables and workspace, so those callers get this single entry point instead.
//
// Its working memory (the fp32 twiddle table and the split-K partial sums of
// the direct kernel) lives in one file-scope __device__ array of
// kScratchBytes.  Every GPU that loads the library holds that array until the
// process exits.  Host code cannot use the array's name as a device address
// (it names a host-side stand-in), so the first call on each device, with that
// device current, looks the address up with cudaGetSymbolAddress and caches
// it; make that first call before any stream capture.  All calls share the
// array and each call rewrites everything it reads (table first, then the
// partials), so nothing needs clearing; calls that overlap on the GPU (other
// streams, other host threads) race on it and must be serialised by the caller.
#include "internal.cuh"

#include <mutex>

namespace ndft {
namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int64_t kMaxNoallocN = 1 << 20;           // fp32 table <= 8 MiB

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

cudaError_t scratch_address(void **out, int *sm_count) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_scratch)) != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    if ((e = cudaDeviceGetAttribute(sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    return cudaSuccess;
}

bool aligned16(const void *ptr) { return ptr && ((uintptr_t)ptr & 15u) == 0; }

}  // namespace
}  // namespace ndft

using namespace ndft;

extern "C" ndft_status caf_exec_noalloc(int32_t n, int32_t p0, int32_t nbins, const void *s_surv, const void *s_ref,
                                        int32_t lag0, int32_t nlags, uint32_t flags, void *A, cudaStream_t stream) {
    if (n < 1 || n > kMaxNoallocN || nbins < 1 || nbins > n || !lag_window_ok(lag0, nlags) || nlags > (1 << 20)) return NDFT_E_INVALID;
    if (flags & ~(uint32_t)(NDFT_F_NO_CONJ_REF | NDFT_F_CIRCULAR_LAG)) return NDFT_E_INVALID;
    if (!aligned16(s_surv) || !aligned16(s_ref) || !aligned16(A)) return NDFT_E_INVALID;
    void *scratch = nullptr;
    int sm = 1;
    if (scratch_address(&scratch, &sm) != cudaSuccess) return NDFT_E_CUDA;

    // scratch layout: [fp32 twiddle table, n float2][split-K partials]
    const size_t table_bytes = (((size_t)n * sizeof(float2)) + 255) & ~(size_t)255;
    const size_t part_room = kScratchBytes - table_bytes;
    const size_t per_split = (size_t)nlags * nbins * sizeof(float2);
    int nsplit = direct_caf_splits(n, nlags, nbins, sm, 0);
    const size_t fit = per_split ? part_room / per_split : 0;
    if ((size_t)nsplit > fit) nsplit = (int)(fit > 0 ? fit : 1);  // one split writes A directly

    Plan p;  // a view onto the scratch array: no allocation
    p.d.n = n;
    p.d.p0 = p0;
    p.d.nbins = nbins;
    p.d.max_lags = nlags;
    p.d.form = NDFT_FORM_DIRECT;
    p.d.prec = NDFT_PREC_FP32;
    p.d.flags = flags;
    p.sm_count = sm;
    p.tw32 = static_cast<float2 *>(scratch);
    p.ws = static_cast<unsigned char *>(scratch) + table_bytes;
    p.ws_bytes = part_room;
    p.tune_split = nsplit;

    cudaError_t e = launch_tables(n, p.tw32, nullptr, stream);
    if (e != cudaSuccess) return NDFT_E_CUDA;
    int launches = 1;
    e = launch_direct_caf(p, s_surv, s_ref, lag0, nlags, A, stream, &launches);
    return e == cudaSuccess ? NDFT_OK : NDFT_E_CUDA;
}
