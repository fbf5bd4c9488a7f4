// plan.cu -- the C ABI of include/ndft.h: argument checks, plan lifecycle,
// dispatch to the kernels.  Exec calls allocate nothing and never synchronise.
#include "internal.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

using namespace ndft;

struct ndft_plan_s {
    Plan p;
};

namespace {

// NVTX range around a C-ABI call (free unless a profiler is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

bool aligned16(const void *ptr) { return ptr && ((uintptr_t)ptr & 15u) == 0; }

// NDFT_LOG=1 in the environment: one line on stderr per plan creation and per
// exec call (what ran and how), read once at the first call.
bool log_on() {
    static const bool on = [] {
        const char *v = std::getenv("NDFT_LOG");
        return v && *v && std::strcmp(v, "0") != 0;
    }();
    return on;
}

void logf(const char *fmt, ...) {
    if (!log_on()) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    std::fprintf(stderr, "[ndft] %s\n", buf);
}

const char *form_name(int f) {
    switch (f) {
        case NDFT_FORM_DIRECT: return "direct";
        case NDFT_FORM_TERNARY_GEMM: return "ternary";
        case NDFT_FORM_NFFT: return "nfft";
        case NDFT_FORM_FFT: return "fft";
    }
    return "?";
}

const char *prec_name(int q) {
    return q == NDFT_PREC_FP32 ? "fp32" : q == NDFT_PREC_BF16X2 ? "bf16x2" : q == NDFT_PREC_Q14 ? "q14" : "?";
}

const char *variant_name(int v) { return v == 2 ? "paired" : v == 1 ? "unpaired" : "-"; }

ndft_status log_exec(const char *what, const Plan &p, int64_t cols, ndft_status st) {
    if (log_on())
        logf("%s N=%d bins=%d@%d cols=%lld form=%s prec=%s variant=%s tile=%d splits=%d launches=%d status=%d", what,
             p.d.n, p.d.nbins, p.d.p0, (long long)cols, form_name(p.d.form), prec_name(p.d.prec),
             variant_name(p.last_variant), p.last_tile, p.last_nsplit, p.last_launches, (int)st);
    return st;
}

thread_local cudaError_t g_last_cuda = cudaSuccess;

ndft_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return NDFT_OK;
    g_last_cuda = e;
    if (e == cudaErrorMemoryAllocation) return NDFT_E_NOMEM;
    return NDFT_E_CUDA;
}

bool pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

bool valid_pair(int form, int prec) {
    if (form == NDFT_FORM_DIRECT) return prec == NDFT_PREC_FP32 || prec == NDFT_PREC_Q14;
    if (form == NDFT_FORM_TERNARY_GEMM) return prec == NDFT_PREC_BF16X2;
    if (form == NDFT_FORM_NFFT || form == NDFT_FORM_FFT) return prec == NDFT_PREC_FP32;
    return false;
}

constexpr uint32_t kKnownFlags =
    NDFT_F_NO_CONJ_REF | NDFT_F_CIRCULAR_LAG | NDFT_F_NFFT_DIF | NDFT_F_Q14_RANGE | NDFT_F_ABS_OUT;

bool fft_form(int form) { return form == NDFT_FORM_NFFT || form == NDFT_FORM_FFT; }
constexpr int32_t kMaxN = 1 << 22;

void free_plan(Plan &p) {
    cudaFree(p.tw32);
    cudaFree(p.twq);
    cudaFree(p.ang);
    cudaFree(p.nfft_ws);
    cudaFree(p.comb);
    cudaFree(p.ws);
    cudaFree(p.atab);
    cudaFree(p.atab_adj);
    std::free(p.tmap_a);
    std::free(p.tmap_a2);
    std::free(p.tmap_adj);
    cudaFree(p.err);
    cudaFree(p.cpis_dev);
    cudaFree(p.tab_arena);
    cudaFree(p.work_dev);
    cudaFree(p.counter);
    cudaFree(p.tmap_dev);
    std::free(p.tmap_host);
    std::free(p.tmap_host2);
    std::free(p.tmap_bpair);
    delete[] p.pair_cpis;
    delete[] p.cpis_host;
    if (p.tev) {
        for (int i = 0; i < 2 * p.tcap; ++i) cudaEventDestroy(p.tev[i]);
        delete[] p.tev;
    }
    if (p.ev_fork) cudaEventDestroy(p.ev_fork);
    if (p.ev_join) cudaEventDestroy(p.ev_join);
    if (p.side) cudaStreamDestroy(p.side);
}

template <class T>
cudaError_t alloc(T **ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void **>(ptr), count * sizeof(T));
}

size_t backward_ws_bytes(const ndft_desc &d) {
    if (d.max_lags <= 0) return 0;
    return (size_t)((d.max_lags + 63) / 64) * d.n * sizeof(float2);
}

int sm_count_now(int *dev) {
    int sm = 0;
    cudaGetDevice(dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, *dev);
    return sm > 0 ? sm : 1;
}

}  // namespace

extern "C" {

const char *ndft_status_string(ndft_status s) {
    switch (s) {
        case NDFT_OK: return "ok";
        case NDFT_E_INVALID: return "invalid argument";
        case NDFT_E_UNSUPPORTED: return "unsupported request";
        case NDFT_E_CUDA: return "CUDA error";
        case NDFT_E_NOMEM: return "out of device memory";
        case NDFT_E_TIMEOUT: return "device-side wait timed out";
        case NDFT_E_OVERFLOW: return "fixed-point overflow";
    }
    return "unknown status";
}

int32_t ndft_version(void) { return 100; }

const char *ndft_last_cuda_error(void) { return cudaGetErrorString(g_last_cuda); }

ndft_status ndft_plan(ndft_plan_t *out, const ndft_desc *d, cudaStream_t stream) {
    const Range range("ndft_plan");
    if (!out || !d) return NDFT_E_INVALID;
    *out = nullptr;
    if (d->n < 1 || d->n > kMaxN || d->nbins < 0 || d->nbins > d->n || d->max_lags < 0 || d->max_batch < 0)
        return NDFT_E_INVALID;
    if (d->max_lags > (1 << 20) || (d->flags & ~kKnownFlags) || d->reserved[0] || d->reserved[1] ||
        d->reserved[2])
        return NDFT_E_INVALID;
    if (!valid_pair(d->form, d->prec)) {
        const bool known = (d->form >= 0 && d->form <= 3) && (d->prec >= 0 && d->prec <= 2);
        return known ? NDFT_E_UNSUPPORTED : NDFT_E_INVALID;
    }
    if ((d->flags & NDFT_F_Q14_RANGE) && d->prec != NDFT_PREC_Q14) return NDFT_E_INVALID;
    if ((d->flags & NDFT_F_ABS_OUT) && d->prec == NDFT_PREC_Q14) return NDFT_E_INVALID;
    if ((d->flags & NDFT_F_ABS_OUT) && fft_form(d->form)) return NDFT_E_UNSUPPORTED;
    if (fft_form(d->form) && (!pow2(d->n) || d->n > 65536)) return NDFT_E_INVALID;
    if (d->form == NDFT_FORM_TERNARY_GEMM && !ternary_supported(*d)) return NDFT_E_UNSUPPORTED;
    auto *h = new (std::nothrow) ndft_plan_s();
    if (!h) return NDFT_E_NOMEM;
    Plan &p = h->p;
    p.d = *d;
    if (p.d.nbins == 0) p.d.nbins = d->n;
    p.sm_count = sm_count_now(&p.device);
    const int N = p.d.n;
    p.g4 = (N % 4 == 0) ? 4 : (N % 2 == 0 ? 2 : 1);
    cudaError_t e = cudaSuccess;
    const bool tern = p.d.form == NDFT_FORM_TERNARY_GEMM;
    if ((e = alloc(&p.tw32, N)) != cudaSuccess) goto fail;
    if (p.d.prec == NDFT_PREC_Q14 && (e = alloc(&p.twq, N)) != cudaSuccess) goto fail;
    if ((e = alloc(&p.err, 1)) != cudaSuccess) goto fail;
    if ((e = cudaMemsetAsync(p.err, 0, sizeof(int32_t), stream)) != cudaSuccess) goto fail;
    p.table_bytes = (size_t)N * (sizeof(float2) + (p.twq ? sizeof(short2) : 0));
    {
        size_t ws = 0;
        if (!fft_form(p.d.form)) ws = std::max(direct_ws_bytes(p.d, p.sm_count), backward_ws_bytes(p.d));
        if (tern) ws = std::max(ws, ternary_ws_bytes(p.d, p.sm_count));
        p.ws_bytes = ws;
        p.ws_alloc = ws;
        if (ws && (e = cudaMalloc(&p.ws, ws)) != cudaSuccess) goto fail;
        const size_t nws = nfft_ws_bytes(p.d, &p.nfft_chunk);
        if (nws && (e = cudaMalloc(&p.nfft_ws, nws)) != cudaSuccess) goto fail;
        p.ws_bytes += nws;
        if (nws && fft_form(p.d.form) && p.d.max_lags > 0) {
            if ((e = alloc(&p.comb, 2 * (size_t)N)) != cudaSuccess) goto fail;
            p.ws_bytes += 2 * (size_t)N * sizeof(float2);
        }
    }
    if ((e = launch_tables(N, p.tw32, p.twq, stream)) != cudaSuccess) goto fail;
    if (tern && (e = ternary_plan_init(p, stream)) != cudaSuccess) goto fail;
    *out = h;
    logf("ndft_plan N=%d bins=%d@%d max_lags=%d max_batch=%lld form=%s prec=%s flags=0x%x bytes=%zu paired_freqs=%d",
         p.d.n, p.d.nbins, p.d.p0, p.d.max_lags, (long long)p.d.max_batch, form_name(p.d.form), prec_name(p.d.prec),
         p.d.flags, p.table_bytes + p.ws_bytes, p.pair_slots);
    return NDFT_OK;
fail:
    free_plan(p);
    delete h;
    cudaGetLastError();  // a failed allocation is also the runtime's last error: do not leak it into later calls
    return from_cuda(e);
}

ndft_status ndft_plan_destroy(ndft_plan_t plan) {
    if (!plan) return NDFT_E_INVALID;
    cudaDeviceSynchronize();
    free_plan(plan->p);
    delete plan;
    return NDFT_OK;
}

ndft_status ndft_exec(ndft_plan_t plan, const void *x, void *X, int64_t batch, cudaStream_t stream) {
    const Range range("ndft_exec");
    if (!plan || plan->p.batched || batch < 0 || batch > plan->p.d.max_batch) return NDFT_E_INVALID;
    Plan &p = plan->p;
    p.last_launches = 0;
    p.last_variant = p.last_nsplit = p.last_tile = 0;
    if (batch == 0) return NDFT_OK;
    if (!aligned16(x) || !aligned16(X) || x == X) return NDFT_E_INVALID;
    if (p.d.flags & NDFT_F_ABS_OUT) return NDFT_E_UNSUPPORTED;
    cudaError_t e;
    if (p.d.form == NDFT_FORM_DIRECT) {
        if (batch > 65535LL * 64) return NDFT_E_UNSUPPORTED;
        e = launch_direct_ndft(p, x, X, batch, stream, &p.last_launches);
    } else if (p.d.form == NDFT_FORM_NFFT) {
        e = launch_nfft_bins(p, x, X, batch, stream, &p.last_launches);
    } else if (p.d.form == NDFT_FORM_FFT) {
        e = launch_fft_bins(p, x, X, batch, stream, &p.last_launches);
    } else {
        e = launch_ternary_ndft(p, x, X, batch, stream, &p.last_launches);
    }
    return log_exec("ndft_exec", p, batch, from_cuda(e));
}

ndft_status nfft_exec(ndft_plan_t plan, const void *x, void *X, int64_t batch, cudaStream_t stream) {
    const Range range("nfft_exec");
    if (!plan || plan->p.batched || batch < 0 || batch > plan->p.d.max_batch) return NDFT_E_INVALID;
    Plan &p = plan->p;
    if (p.d.prec != NDFT_PREC_FP32 || !pow2(p.d.n) || p.d.n > (1 << 20) || p.d.nbins != p.d.n ||
        p.d.p0 % p.d.n != 0)
        return NDFT_E_INVALID;
    if ((p.d.flags & NDFT_F_NFFT_DIF) && p.d.n > 65536) return NDFT_E_UNSUPPORTED;
    p.last_launches = 0;
    p.last_variant = p.last_nsplit = p.last_tile = 0;
    if (batch == 0) return NDFT_OK;
    if (!aligned16(x) || !aligned16(X)) return NDFT_E_INVALID;
    return log_exec("nfft_exec", p, batch, from_cuda(launch_nfft(p, x, X, batch, stream, &p.last_launches)));
}

ndft_status caf_exec(ndft_plan_t plan, const void *s_surv, const void *s_ref, int32_t lag0, int32_t nlags, void *A,
                     cudaStream_t stream) {
    const Range range("caf_exec");
    if (!plan || plan->p.batched || !lag_window_ok(lag0, nlags) || nlags > plan->p.d.max_lags) return NDFT_E_INVALID;
    if (!aligned16(s_surv) || !aligned16(s_ref) || !aligned16(A)) return NDFT_E_INVALID;
    if (A == s_surv || A == s_ref) return NDFT_E_INVALID;
    Plan &p = plan->p;
    p.last_launches = 0;
    p.last_variant = p.last_nsplit = p.last_tile = 0;
    cudaError_t e;
    if (p.d.form == NDFT_FORM_DIRECT)
        e = launch_direct_caf(p, s_surv, s_ref, lag0, nlags, A, stream, &p.last_launches);
    else if (p.d.form == NDFT_FORM_NFFT)
        e = launch_nfft_caf(p, s_surv, s_ref, lag0, nlags, A, stream, &p.last_launches);
    else if (p.d.form == NDFT_FORM_FFT)
        e = launch_fft_caf(p, s_surv, s_ref, lag0, nlags, A, stream, &p.last_launches);
    else
        e = launch_ternary_caf(p, s_surv, s_ref, lag0, nlags, A, stream, &p.last_launches);
    return log_exec("caf_exec", p, nlags, from_cuda(e));
}

ndft_status caf_backward(ndft_plan_t plan, const void *s_surv, const void *s_ref, int32_t lag0, int32_t nlags,
                         const void *dA, void *ds, cudaStream_t stream) {
    const Range range("caf_backward");
    (void)s_surv;
    if (!plan || plan->p.batched || !lag_window_ok(lag0, nlags) || nlags > plan->p.d.max_lags) return NDFT_E_INVALID;
    Plan &p = plan->p;
    if (p.d.prec == NDFT_PREC_Q14 || fft_form(p.d.form)) return NDFT_E_UNSUPPORTED;
    if (!aligned16(s_ref) || !aligned16(dA) || !aligned16(ds)) return NDFT_E_INVALID;
    if (ds == s_ref || ds == dA) return NDFT_E_INVALID;
    p.last_launches = 0;
    p.last_variant = p.last_nsplit = p.last_tile = 0;
    if (p.d.form == NDFT_FORM_TERNARY_GEMM) {
        // the transposed ternary contraction on the tensor cores (CUDA cores if it does not fit)
        const cudaError_t e = launch_ternary_adjoint(p, s_ref, lag0, nlags, dA, ds, stream, &p.last_launches);
        if (e != cudaErrorNotSupported) return from_cuda(e);
        p.last_launches = 0;
    p.last_variant = p.last_nsplit = p.last_tile = 0;
    }
    return from_cuda(launch_caf_backward(p, s_ref, lag0, nlags, dA, ds, stream, &p.last_launches));
}

ndft_status caf_backward_inputs(ndft_plan_t plan, const void *s_surv, const void *s_ref, int32_t lag0,
                                int32_t nlags, const void *dA, void *ds_surv, void *ds_ref, cudaStream_t stream) {
    if (!ds_ref) return ds_surv ? caf_backward(plan, s_surv, s_ref, lag0, nlags, dA, ds_surv, stream) : NDFT_E_INVALID;
    const Range range("caf_backward_inputs");
    if (!plan || plan->p.batched || !lag_window_ok(lag0, nlags) || nlags > plan->p.d.max_lags) return NDFT_E_INVALID;
    Plan &p = plan->p;
    if (p.d.prec == NDFT_PREC_Q14 || fft_form(p.d.form)) return NDFT_E_UNSUPPORTED;
    if (!aligned16(s_surv) || !aligned16(s_ref) || !aligned16(dA) || !aligned16(ds_ref) ||
        (ds_surv && !aligned16(ds_surv)))
        return NDFT_E_INVALID;
    if (ds_ref == s_surv || ds_ref == s_ref || ds_ref == dA || ds_surv == ds_ref || ds_surv == s_surv ||
        ds_surv == s_ref || ds_surv == dA)
        return NDFT_E_INVALID;  // the fold reads both inputs while it writes the gradients
    p.last_launches = 0;
    p.last_variant = p.last_nsplit = p.last_tile = 0;
    const cudaError_t e =
        launch_caf_backward_inputs(p, s_surv, s_ref, lag0, nlags, dA, ds_surv, ds_ref, stream, &p.last_launches);
    if (e == cudaErrorNotSupported) return NDFT_E_UNSUPPORTED;
    return from_cuda(e);
}

ndft_status ndft_argmax(const void *X, int64_t rows, int64_t cols, int64_t *idx, float *val, cudaStream_t stream) {
    if (rows < 0 || cols < 1 || (rows > 0 && (!X || !idx))) return NDFT_E_INVALID;
    if (((uintptr_t)X & 7u) || ((uintptr_t)idx & 7u) || ((uintptr_t)val & 3u)) return NDFT_E_INVALID;
    return from_cuda(launch_argmax(static_cast<const float2 *>(X), rows, cols, idx, val, stream));
}

ndft_status ndft_query_error(ndft_plan_t plan, cudaStream_t stream) {
    if (!plan) return NDFT_E_INVALID;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return NDFT_E_CUDA;
    int32_t v = 0;
    if ((e = cudaMemcpy(&v, plan->p.err, sizeof(v), cudaMemcpyDeviceToHost)) != cudaSuccess) return NDFT_E_CUDA;
    if (v != 0 && (e = cudaMemset(plan->p.err, 0, sizeof(int32_t))) != cudaSuccess) return NDFT_E_CUDA;
    if (v == 0) return NDFT_OK;
    if (v == kDevTimeout) return NDFT_E_TIMEOUT;
    if (v == kDevOverflow) return NDFT_E_OVERFLOW;
    return NDFT_E_CUDA;
}

ndft_status ndft_get_twiddles(ndft_plan_t plan, int32_t which, void *dst, cudaStream_t stream) {
    if (!plan || plan->p.batched || !dst) return NDFT_E_INVALID;
    const Plan &p = plan->p;
    const int N = p.d.n;
    const void *src = nullptr;
    size_t bytes = 0;
    if (which == 0) {
        src = p.tw32;
        bytes = (size_t)N * sizeof(float2);
    } else if (which == 1) {
        src = p.twq;
        bytes = (size_t)N * sizeof(short2);
    } else if (which == 2) {
        src = p.ang;
        bytes = (size_t)((N - 1) / 256 + 1 + 256) * sizeof(float2);
    } else {
        return NDFT_E_INVALID;
    }
    if (!src) return NDFT_E_UNSUPPORTED;
    return from_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, stream));
}

ndft_status ndft_plan_bytes(ndft_plan_t plan, int64_t *bytes) {
    if (!plan || !bytes) return NDFT_E_INVALID;
    *bytes = (int64_t)(plan->p.table_bytes + plan->p.ws_bytes);
    return NDFT_OK;
}

ndft_status ndft_last_launches(ndft_plan_t plan, int32_t *count) {
    if (!plan || !count) return NDFT_E_INVALID;
    *count = plan->p.last_launches;
    return NDFT_OK;
}

ndft_status ndft_timer_start(ndft_plan_t plan, int32_t capacity) {
    if (!plan || capacity < 0 || capacity > (1 << 20)) return NDFT_E_INVALID;
    Plan &p = plan->p;
    if (p.tev) {
        cudaDeviceSynchronize();
        for (int i = 0; i < 2 * p.tcap; ++i) cudaEventDestroy(p.tev[i]);
        delete[] p.tev;
        p.tev = nullptr;
        p.tcap = p.tcount = 0;
    }
    if (capacity == 0) return NDFT_OK;
    p.tev = new (std::nothrow) cudaEvent_t[2 * capacity];
    if (!p.tev) return NDFT_E_NOMEM;
    for (int i = 0; i < 2 * capacity; ++i) {
        if (cudaEventCreate(&p.tev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(p.tev[j]);
            delete[] p.tev;
            p.tev = nullptr;
            return NDFT_E_CUDA;
        }
    }
    p.tcap = capacity;
    p.tcount = 0;
    return NDFT_OK;
}

ndft_status ndft_timer_read(ndft_plan_t plan, double *ms_total, int32_t *count) {
    if (!plan || !ms_total || !count) return NDFT_E_INVALID;
    Plan &p = plan->p;
    double tot = 0.0;
    for (int i = 0; i < p.tcount; ++i) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.tev[2 * i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, p.tev[2 * i], p.tev[2 * i + 1]) != cudaSuccess)
            return NDFT_E_CUDA;
        tot += ms;
    }
    *ms_total = tot;
    *count = p.tcount;
    p.tcount = 0;
    return NDFT_OK;
}

ndft_status ndft_plan_query(ndft_plan_t plan, int32_t key, int64_t *value) {
    if (!plan || !value) return NDFT_E_INVALID;
    const Plan &p = plan->p;
    if (key == 0) *value = p.pair_slots;
    else if (key == 1) *value = p.last_variant;
    else if (key == 2) *value = p.last_nsplit;
    else if (key == 3) *value = p.last_tile;
    else return NDFT_E_INVALID;
    return NDFT_OK;
}

ndft_status ndft_set_tuning(ndft_plan_t plan, int32_t key, int32_t value) {
    if (!plan || value < 0) return NDFT_E_INVALID;
    if (key == 0) {
        if (value > 4096) return NDFT_E_INVALID;
        plan->p.tune_split = value;
    } else if (key == 1) {
        if (value != 0 && value != 128 && value != 256 && value != 258) return NDFT_E_INVALID;
        plan->p.tune_cols = value;
    } else if (key == 2) {
        if (value > 1 << 20) return NDFT_E_INVALID;
        plan->p.tune_chunk = value;
    } else if (key == 3) {
        if (value > 1) return NDFT_E_INVALID;
        plan->p.tune_drain = value;
    } else if (key == 4) {
        if (value > 1) return NDFT_E_INVALID;
        plan->p.test_starve = value;
    } else if (key == 5) {
        if (value > (1 << 20) || (value > 1 && value % 256)) return NDFT_E_INVALID;
        plan->p.tune_parts = value;
    } else if (key == 6) {
        if (value > 2) return NDFT_E_INVALID;
        plan->p.tune_pair = value;
    } else if (key == 7) {
        if (value > 1) return NDFT_E_INVALID;
        plan->p.tune_atab = value;
    } else if (key == 8) {
        if (value > 3) return NDFT_E_INVALID;
        plan->p.tune_bgen = value;
    } else if (key == 9) {
        if (value > 64) return NDFT_E_INVALID;
        plan->p.tune_look = value;
    } else if (key == 10) {
        if (value > 2) return NDFT_E_INVALID;
        plan->p.tune_adj_atab = value;
    } else {
        return NDFT_E_INVALID;
    }
    return NDFT_OK;
}

// ---- batched plans -----------------------------------------------------------------

ndft_status ndft_plan_batched(ndft_plan_t *out, const ndft_cpi *cpis, int32_t ncpi, int32_t form, int32_t prec,
                              uint32_t flags, cudaStream_t stream) {
    const Range range("ndft_plan_batched");
    if (!out || !cpis || ncpi < 1 || ncpi > (1 << 20) || (flags & ~kKnownFlags)) return NDFT_E_INVALID;
    if ((flags & NDFT_F_Q14_RANGE) && prec != NDFT_PREC_Q14) return NDFT_E_INVALID;
    if (flags & NDFT_F_ABS_OUT) return NDFT_E_UNSUPPORTED;
    *out = nullptr;
    if (!valid_pair(form, prec) || fft_form(form)) return NDFT_E_UNSUPPORTED;
    for (int c = 0; c < ncpi; ++c) {
        const ndft_cpi &q = cpis[c];
        if (q.n < 1 || q.n > kMaxN || !lag_window_ok(q.lag0, q.nlags) || q.nlags > (1 << 20) || q.nbins < 1 || q.nbins > q.n ||
            q.off_surv < 0 || q.off_ref < 0 || q.off_out < 0 || q.reserved)
            return NDFT_E_INVALID;
        // 16-byte alignment of each CPI's rows: offsets in elements of 8 bytes (complex64) or 4 (Q1.14)
        const int esz = prec == NDFT_PREC_Q14 ? 4 : 8;
        if ((q.off_surv * esz) % 16 || (q.off_ref * esz) % 16) return NDFT_E_INVALID;
        if (form == NDFT_FORM_TERNARY_GEMM) {
            ndft_desc one{};
            one.n = q.n;
            one.form = form;
            one.prec = prec;
            if (!ternary_supported(one)) return NDFT_E_UNSUPPORTED;
        }
    }
    auto *h = new (std::nothrow) ndft_plan_s();
    if (!h) return NDFT_E_NOMEM;
    Plan &p = h->p;
    p.batched = true;
    p.d = ndft_desc{};
    p.d.form = form;
    p.d.prec = prec;
    p.d.flags = flags;
    p.ncpi = ncpi;
    p.sm_count = sm_count_now(&p.device);
    cudaError_t e = cudaSuccess;
    std::vector<int32_t> work;
    if (form == NDFT_FORM_TERNARY_GEMM) {
        if ((e = alloc(&p.err, 1)) != cudaSuccess || (e = cudaMemsetAsync(p.err, 0, sizeof(int32_t), stream)) != cudaSuccess ||
            (e = ternary_batched_init(p, cpis, ncpi, stream)) != cudaSuccess) {
            free_plan(p);
            delete h;
            return e == cudaErrorNotSupported ? NDFT_E_UNSUPPORTED : from_cuda(e);
        }
        *out = h;
        return NDFT_OK;
    }
    p.cpis_host = new (std::nothrow) CpiDev[ncpi];
    if (!p.cpis_host) {
        delete h;
        return NDFT_E_NOMEM;
    }
    {
        const size_t tsz = prec == NDFT_PREC_Q14 ? sizeof(short2) : sizeof(float2);
        int64_t tw_total = 0;
        for (int c = 0; c < ncpi; ++c) {
            CpiDev &q = p.cpis_host[c];
            std::memset(&q, 0, sizeof(q));
            q.off_surv = cpis[c].off_surv;
            q.off_ref = cpis[c].off_ref;
            q.off_out = cpis[c].off_out;
            q.n = cpis[c].n;
            q.lag0 = cpis[c].lag0;
            q.nlags = cpis[c].nlags;
            q.p0 = cpis[c].p0;
            q.nbins = cpis[c].nbins;
            q.tab = c;
            q.tw_off = tw_total;
            tw_total += (q.n + 3) & ~3;  // keep every table 16-byte aligned
        }
        if ((e = cudaMalloc(&p.tab_arena, std::max<size_t>(16, tw_total * tsz))) != cudaSuccess) goto fail;
        p.table_bytes = tw_total * tsz;
        for (int c = 0; c < ncpi; ++c) {
            const CpiDev &q = p.cpis_host[c];
            float2 *t32 = prec == NDFT_PREC_Q14 ? nullptr : static_cast<float2 *>(p.tab_arena) + q.tw_off;
            short2 *tq = prec == NDFT_PREC_Q14 ? static_cast<short2 *>(p.tab_arena) + q.tw_off : nullptr;
            if ((e = launch_tables(q.n, t32, tq, stream)) != cudaSuccess) goto fail;
        }
        // work list: (cpi, bin tile, lag tile), longest CPIs first
        std::vector<int> order(ncpi);
        for (int c = 0; c < ncpi; ++c) order[c] = c;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (int64_t)p.cpis_host[a].n > (int64_t)p.cpis_host[b].n;
        });
        for (int c : order) {
            const CpiDev &q = p.cpis_host[c];
            for (int bt = 0; bt < (q.nbins + 63) / 64; ++bt)
                for (int lt = 0; lt < (q.nlags + 63) / 64; ++lt) {
                    work.push_back(c);
                    work.push_back(bt);
                    work.push_back(lt);
                }
        }
        p.nwork = (int64_t)work.size() / 3;
        if ((e = alloc(&p.work_dev, work.size())) != cudaSuccess) goto fail;
        if ((e = cudaMemcpyAsync(p.work_dev, work.data(), work.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 stream)) != cudaSuccess)
            goto fail;
        if ((e = alloc(&p.cpis_dev, ncpi)) != cudaSuccess) goto fail;
        if ((e = cudaMemcpyAsync(p.cpis_dev, p.cpis_host, ncpi * sizeof(CpiDev), cudaMemcpyHostToDevice, stream)) !=
            cudaSuccess)
            goto fail;
        if ((e = alloc(&p.counter, 1)) != cudaSuccess) goto fail;
        if ((e = alloc(&p.err, 1)) != cudaSuccess) goto fail;
        if ((e = cudaMemsetAsync(p.err, 0, sizeof(int32_t), stream)) != cudaSuccess) goto fail;
        // the host vector must outlive the async copy
        if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) goto fail;
    }
    *out = h;
    return NDFT_OK;
fail:
    free_plan(p);
    delete h;
    cudaGetLastError();  // a failed allocation is also the runtime's last error: do not leak it into later calls
    return from_cuda(e);
}

ndft_status caf_exec_batched(ndft_plan_t plan, const void *surv_base, const void *ref_base, void *out_base,
                             cudaStream_t stream) {
    const Range range("caf_exec_batched");
    if (!plan || !plan->p.batched) return NDFT_E_INVALID;
    if (!aligned16(surv_base) || !aligned16(ref_base) || !aligned16(out_base)) return NDFT_E_INVALID;
    if (out_base == surv_base || out_base == ref_base) return NDFT_E_INVALID;
    Plan &p = plan->p;
    p.last_launches = 0;
    p.last_variant = p.last_nsplit = p.last_tile = 0;
    if (p.d.form == NDFT_FORM_TERNARY_GEMM) {
        const cudaError_t e = launch_ternary_batched(p, surv_base, ref_base, out_base, stream, &p.last_launches);
        return e == cudaErrorNotSupported ? NDFT_E_UNSUPPORTED : from_cuda(e);
    }
    return from_cuda(launch_direct_batched(p, surv_base, ref_base, out_base, stream, &p.last_launches));
}

}  // extern "C"
