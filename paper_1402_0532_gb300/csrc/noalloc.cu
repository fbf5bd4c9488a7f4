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
// it together with the device's current context; the same set-up also loads
// every kernel the call can launch (the table kernel, the direct CAF kernel
// and the split sum), so that later calls load no module.  Make that first
// call before any stream capture.  A device whose context was reset
// (cudaDeviceReset) gets a new context, and the next call repeats the set-up:
// make it before any capture as well.  All calls share the array and each
// call rewrites everything it reads (table first, then the partials), so
// nothing needs clearing; calls that overlap on the GPU (other streams, other
// host threads) race on it and must be serialised by the caller.
#include "internal.cuh"

#include <cuda.h>

#include <mutex>

namespace ndft {
namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int64_t kMaxNoallocN = 1 << 20;           // fp32 table <= 8 MiB

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];
CUcontext g_scratch_ctx[kMaxDevices];
std::mutex g_scratch_mu;

// The calling thread's current context, through the runtime's driver entry
// point (the library does not link the driver library itself).
cudaError_t current_context(CUcontext *ctx) {
    using Fn = CUresult (*)(CUcontext *);
    static Fn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return cudaErrorNotSupported;
        fn = reinterpret_cast<Fn>(p);
    }
    return fn(ctx) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

cudaError_t scratch_address(void **out, int *sm_count) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    CUcontext ctx = nullptr;  // NULL before the runtime has set up a context on this thread
    if ((e = current_context(&ctx)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!ctx || !g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_scratch)) != cudaSuccess) return e;
        if ((e = tables_preload()) != cudaSuccess) return e;
        if ((e = direct_caf_preload()) != cudaSuccess) return e;
        if ((e = reduce_preload()) != cudaSuccess) return e;
        if ((e = current_context(&ctx)) != cudaSuccess) return e;  // set up by the lookup if it was not
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
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
