"""Thin PyTorch binding over the C ABI (include/ndft.h).

PyTorch provides device memory and the current stream; every step of the
transforms runs in the library's CUDA kernels.  Each method marshals tensor
pointers into the C call of the same name and raises ``NdftError`` on a
non-OK status.  Inputs must be CUDA tensors: there is no CPU path.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from ._lib import F_ABS_OUT, F_CIRCULAR_LAG, F_NFFT_DIF, F_NO_CONJ_REF, F_Q14_RANGE  # noqa: F401  (plan flags)

_FORMS = {"direct": L.FORM_DIRECT, "ternary": L.FORM_TERNARY_GEMM, "nfft": L.FORM_NFFT, "fft": L.FORM_FFT}
_PRECS = {"fp32": L.PREC_FP32, "bf16x2": L.PREC_BF16X2, "q14": L.PREC_Q14}


def choose_form(n: int) -> tuple[str, str]:
    """(form, prec) of the faster exact-⊗ evaluation of Eq. 8 / Eq. 12a for
    N = n samples, by the measured crossover on one GB300 (NDFT batches of
    16..4096 columns, 32..1024 bins, N = 64..16384): the plain form on the CUDA
    cores for N <= 64 (there the tensor-core form's packing and launch costs
    dominate: 0.021 against 0.027 ms for 4096 vectors), the tensor-core form
    everywhere else (from ties at N = 256 to 33x at N = 16384).  Both meet the
    same 1e-5 bar; for bit-reproducible integer results use prec="q14" with
    the plain form."""
    return ("direct", "fp32") if int(n) <= 64 else ("ternary", "bf16x2")


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _need(t: torch.Tensor, dtype, what: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor (the library has no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A single-transform plan: ``ndft``, ``nfft``, ``caf``, ``caf_backward``.

    form: "direct" (CUDA cores), "ternary" (tcgen05 tensor cores), "nfft"
    (the Sec. 3 NFFT in place of the NDFT: ``ndft`` gives NFFT bins, ``caf``
    Eq. 12a through the NFFT) or "fft" (the ordinary DFT by an fp32 FFT:
    ``ndft`` gives DFT bins, ``caf`` Eq. 12b); nfft/fft need N a power of two
    <= 65536.  flags: F_NO_CONJ_REF, F_CIRCULAR_LAG, F_NFFT_DIF (decimation in
    frequency for ``nfft`` and the nfft form);
    prec: "fp32" / "q14" (direct), "bf16x2" (ternary), "fp32" (nfft, fft).
    form="auto" takes the form and precision ``choose_form(n)`` names (prec is
    then ignored).  Bins are p0 .. p0 + nbins - 1 (nbins = 0 -> N)."""

    def __init__(self, n: int, *, p0: int = 0, nbins: int = 0, max_lags: int = 0, max_batch: int = 0,
                 form: str = "direct", prec: str = "fp32", flags: int = 0, device=None):
        if form == "auto":
            form, prec = choose_form(n)
        self.lib = L.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.n, self.p0 = int(n), int(p0)
        self.nbins = int(nbins) if nbins else int(n)
        self.max_lags, self.max_batch = int(max_lags), int(max_batch)
        self.form, self.prec, self.flags = form, prec, int(flags)
        self._args = dict(p0=p0, nbins=nbins, max_lags=max_lags, max_batch=max_batch, form=form, prec=prec,
                          flags=flags, device=self.device)
        self._tuning = {}
        d = L.NdftDesc(n=self.n, p0=self.p0, nbins=int(nbins), max_lags=self.max_lags,
                       max_batch=self.max_batch, form=_FORMS[form], prec=_PRECS[prec], flags=self.flags)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            L.check(self.lib.ndft_plan(ctypes.byref(h), ctypes.byref(d), _stream(self.device)), "ndft_plan")
        self.handle = h

    # -- helpers -----------------------------------------------------------------
    @property
    def _in_dtype(self):
        return torch.int16 if self.prec == "q14" else torch.complex64

    @property
    def _out_dtype(self):
        return torch.int32 if self.prec == "q14" else torch.complex64

    def _row_shape(self, n):
        return (n, 2) if self.prec == "q14" else (n,)

    def close(self):
        if getattr(self, "handle", None):
            L.check(self.lib.ndft_plan_destroy(self.handle), "ndft_plan_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_launches(self) -> int:
        c = ctypes.c_int32()
        L.check(self.lib.ndft_last_launches(self.handle, ctypes.byref(c)), "ndft_last_launches")
        return c.value

    def nbytes(self) -> int:
        b = ctypes.c_int64()
        L.check(self.lib.ndft_plan_bytes(self.handle, ctypes.byref(b)), "ndft_plan_bytes")
        return b.value

    def set_tuning(self, key: int, value: int):
        L.check(self.lib.ndft_set_tuning(self.handle, int(key), int(value)), "ndft_set_tuning")
        self._tuning[int(key)] = int(value)

    def query(self, key: int) -> int:
        """ndft_plan_query: 0 = paired frequencies S of the window, 1 = last call's
        contraction variant (0 none, 1 unpaired rows, 2 conjugate-paired rows),
        2 = last call's sample-axis split count, 3 = its tile (256 / 128 rows on
        one CTA, 258 the 2-SM pair)."""
        v = ctypes.c_int64()
        L.check(self.lib.ndft_plan_query(self.handle, int(key), ctypes.byref(v)), "ndft_plan_query")
        return v.value

    def twin(self) -> "Plan":
        """A second plan with this plan's descriptor and tuning settings and its own
        tables and workspace: same results bit for bit, and the two can run at once on
        two streams."""
        t = Plan(self.n, **self._args)
        for k, v in self._tuning.items():
            t.set_tuning(k, v)
        return t

    def timer_start(self, capacity: int):
        """Arm device timing of the main kernel for the next `capacity` exec calls."""
        L.check(self.lib.ndft_timer_start(self.handle, int(capacity)), "ndft_timer_start")

    def timer_read(self) -> tuple[float, int]:
        """(summed milliseconds, launches timed) of the main kernel since timer_start / the last read."""
        ms, n = ctypes.c_double(), ctypes.c_int32()
        L.check(self.lib.ndft_timer_read(self.handle, ctypes.byref(ms), ctypes.byref(n)), "ndft_timer_read")
        return ms.value, n.value

    def query_error(self):
        L.check(self.lib.ndft_query_error(self.handle, _stream(self.device)), "ndft_query_error")

    def twiddles(self, which: int = 0) -> torch.Tensor:
        """The plan's table: 0 fp32 twiddles [N] complex64, 1 Q1.14 twiddles [N, 2] int16,
        2 the ternary form's two-level (cos, sin) table [(N-1)//256 + 1 + 256] complex64."""
        n = self.n
        if which == 0:
            out = torch.empty(n, dtype=torch.complex64, device=self.device)
        elif which == 1:
            out = torch.empty(n, 2, dtype=torch.int16, device=self.device)
        else:
            out = torch.empty((n - 1) // 256 + 1 + 256, dtype=torch.complex64, device=self.device)
        L.check(self.lib.ndft_get_twiddles(self.handle, int(which), _ptr(out), _stream(self.device)),
                "ndft_get_twiddles")
        return out

    # -- transforms ----------------------------------------------------------------
    def ndft(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Eq. 8 over the rows of x ([batch, N] complex64, or [batch, N, 2] int16 for q14)."""
        _need(x, self._in_dtype, "x")
        batch = x.shape[0]
        if out is None:
            out = torch.empty((batch,) + self._row_shape(self.nbins), dtype=self._out_dtype, device=x.device)
        _need(out, self._out_dtype, "out")
        L.check(self.lib.ndft_exec(self.handle, _ptr(x), _ptr(out), batch, _stream(x.device)), "ndft_exec")
        return out

    def nfft(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Sec. 3 NFFT over the rows of x ([batch, N] complex64); out may be x."""
        _need(x, torch.complex64, "x")
        if out is None:
            out = torch.empty_like(x)
        _need(out, torch.complex64, "out")
        L.check(self.lib.nfft_exec(self.handle, _ptr(x), _ptr(out), x.shape[0], _stream(x.device)), "nfft_exec")
        return out

    def caf(self, s_surv: torch.Tensor, s_ref: torch.Tensor, lag0: int, nlags: int,
            out: torch.Tensor | None = None) -> torch.Tensor:
        """Eq. 12a surface [nlags, nbins] (complex64, [nlags, nbins, 2] int32 for q14, or the
        magnitudes [nlags, nbins] float32 on plans with F_ABS_OUT)."""
        _need(s_surv, self._in_dtype, "s_surv")
        _need(s_ref, self._in_dtype, "s_ref")
        odt = torch.float32 if self.flags & F_ABS_OUT else self._out_dtype
        if out is None:
            out = torch.empty((nlags,) + self._row_shape(self.nbins), dtype=odt, device=s_surv.device)
        _need(out, odt, "out")
        L.check(self.lib.caf_exec(self.handle, _ptr(s_surv), _ptr(s_ref), int(lag0), int(nlags), _ptr(out),
                                  _stream(s_surv.device)), "caf_exec")
        return out

    def caf_from_host(self, s_surv_host: torch.Tensor, s_ref_host: torch.Tensor, lag0: int, nlags: int,
                      out_host: torch.Tensor, staging: dict | None = None) -> torch.Tensor:
        """caf() for host (ideally pinned) buffers: copies the inputs to the device, runs
        caf_exec and copies the surface back, all on the current stream; synchronises.
        `staging` (optional dict) keeps the device buffers between calls."""
        st = {} if staging is None else staging
        if "ss" not in st:
            st["ss"] = torch.empty_like(s_surv_host, device=self.device)
            st["sr"] = torch.empty_like(s_ref_host, device=self.device)
            st["A"] = torch.empty((nlags,) + self._row_shape(self.nbins), dtype=self._out_dtype, device=self.device)
        st["ss"].copy_(s_surv_host, non_blocking=True)
        st["sr"].copy_(s_ref_host, non_blocking=True)
        self.caf(st["ss"], st["sr"], lag0, nlags, out=st["A"])
        out_host.copy_(st["A"], non_blocking=True)
        torch.cuda.current_stream(self.device).synchronize()
        return out_host

    def caf_from_host_many(self, inputs, lag0: int, nlags: int, outs, staging: dict | None = None,
                           overlap: bool = False):
        """caf_from_host over a sequence of (s_surv_host, s_ref_host) pairs into the host
        surfaces `outs` (one per pair, or one buffer reused), pipelined: two device buffer
        sets, the inputs of step k copied in on one stream while step k - 1 computes, and
        the surface of step k - 1 copied out on another while step k computes.  Every step
        still copies its inputs in and its surface out.  overlap=False: every step computes
        on the current stream with this plan.  overlap=True: odd steps compute on a second
        stream with a twin plan (``twin()``, kept in `staging`; its own workspace, about
        ``nbytes()`` more device memory), so the surfaces of consecutive steps can overlap
        on the GPU (the lag-product packing of step k under the contraction of step k - 1);
        the surfaces are the same bit for bit.  Synchronises before returning."""
        st = {} if staging is None else staging
        dev = self.device
        comp = torch.cuda.current_stream(dev)
        if "h2d" not in st:
            st["h2d"], st["d2h"] = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        inputs = list(inputs)
        if not inputs:
            return outs
        if overlap:
            if "twin" not in st:
                st["twin"], st["comp2"] = self.twin(), torch.cuda.Stream(dev)
            for k, v in self._tuning.items():  # follow tuning changes made since the twin was made
                if st["twin"]._tuning.get(k) != v:
                    st["twin"].set_tuning(k, v)
            plans, comps = (self, st["twin"]), (comp, st["comp2"])
            st["comp2"].wait_stream(comp)
        else:
            plans, comps = (self, self), (comp, comp)
        hs0, hr0 = inputs[0]
        if "pipe" not in st:
            st["pipe"] = [dict(ss=torch.empty_like(hs0, device=dev), sr=torch.empty_like(hr0, device=dev),
                               A=torch.empty((nlags,) + self._row_shape(self.nbins), dtype=self._out_dtype,
                                             device=dev)) for _ in range(2)]
        bufs = st["pipe"]
        ev = lambda: torch.cuda.Event()  # noqa: E731
        e_in, e_comp, e_out = [ev(), ev()], [None, None], [None, None]
        single_out = not isinstance(outs, (list, tuple))
        for k, (hs, hr) in enumerate(inputs):
            b = k % 2
            buf, cs = bufs[b], comps[b]
            with torch.cuda.stream(st["h2d"]):
                if e_comp[b] is not None:
                    st["h2d"].wait_event(e_comp[b])  # step k - 2 is done reading this buffer
                buf["ss"].copy_(hs, non_blocking=True)
                buf["sr"].copy_(hr, non_blocking=True)
                e_in[b].record(st["h2d"])
            cs.wait_event(e_in[b])
            if e_out[b] is not None:
                cs.wait_event(e_out[b])  # the surface of step k - 2 has been copied out
            with torch.cuda.stream(cs):
                plans[b].caf(buf["ss"], buf["sr"], lag0, nlags, out=buf["A"])
            e_comp[b] = ev()
            e_comp[b].record(cs)
            with torch.cuda.stream(st["d2h"]):
                st["d2h"].wait_event(e_comp[b])
                (outs if single_out else outs[k]).copy_(buf["A"], non_blocking=True)
                e_out[b] = ev()
                e_out[b].record(st["d2h"])
        st["d2h"].synchronize()
        for cs in comps:
            cs.synchronize()
        if overlap:
            comp.wait_stream(st["comp2"])
            st["twin"].query_error()
        return outs

    def caf_backward(self, s_surv: torch.Tensor, s_ref: torch.Tensor, lag0: int, nlags: int, dA: torch.Tensor,
                     out: torch.Tensor | None = None) -> torch.Tensor:
        """dL/ds_surv (dRe + j dIm) given dA = dL/dRe A + j dL/dIm A ([nlags, nbins] complex64)."""
        _need(s_ref, torch.complex64, "s_ref")
        _need(dA, torch.complex64, "dA")
        if out is None:
            out = torch.empty(self.n, dtype=torch.complex64, device=s_ref.device)
        _need(out, torch.complex64, "out")
        L.check(self.lib.caf_backward(self.handle, _ptr(s_surv), _ptr(s_ref), int(lag0), int(nlags), _ptr(dA),
                                      _ptr(out), _stream(s_ref.device)), "caf_backward")
        return out


    def caf_backward_inputs(self, s_surv: torch.Tensor, s_ref: torch.Tensor, lag0: int, nlags: int,
                            dA: torch.Tensor, surv: bool = True):
        """(dL/ds_surv or None, dL/ds_ref), each dRe + j dIm, from one adjoint contraction."""
        _need(s_surv, torch.complex64, "s_surv")
        _need(s_ref, torch.complex64, "s_ref")
        _need(dA, torch.complex64, "dA")
        ds_ref = torch.empty(self.n, dtype=torch.complex64, device=s_ref.device)
        ds_surv = torch.empty(self.n, dtype=torch.complex64, device=s_ref.device) if surv else None
        L.check(self.lib.caf_backward_inputs(self.handle, _ptr(s_surv), _ptr(s_ref), int(lag0), int(nlags),
                                             _ptr(dA), _ptr(ds_surv) if surv else None, _ptr(ds_ref),
                                             _stream(s_ref.device)), "caf_backward_inputs")
        return ds_surv, ds_ref

class BatchedPlan:
    """caf_exec_batched over a fixed list of CPIs (one persistent launch sequence).

    cpis: list of dicts with keys off_surv, off_ref, off_out, n, lag0, nlags, p0, nbins."""

    def __init__(self, cpis, *, form: str = "direct", prec: str = "fp32", flags: int = 0):
        self.lib = L.load()
        self.device = torch.device("cuda", torch.cuda.current_device())
        arr = (L.NdftCpi * len(cpis))()
        for i, c in enumerate(cpis):
            arr[i] = L.NdftCpi(off_surv=c["off_surv"], off_ref=c["off_ref"], off_out=c["off_out"], n=c["n"],
                               lag0=c["lag0"], nlags=c["nlags"], p0=c["p0"], nbins=c["nbins"])
        self.form, self.prec = form, prec
        # a short digest of the CPI list, for the autotuner's cache key
        import hashlib
        shape = ";".join(f"{c['n']},{c['nlags']},{c['nbins']}" for c in cpis)
        self._sig = f"{len(cpis)}cpis-" + hashlib.sha1(shape.encode()).hexdigest()[:12]
        h = ctypes.c_void_p()
        L.check(self.lib.ndft_plan_batched(ctypes.byref(h), arr, len(cpis), _FORMS[form], _PRECS[prec], int(flags),
                                           _stream(self.device)), "ndft_plan_batched")
        self.handle = h

    def __call__(self, surv: torch.Tensor, ref: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
        dt_in = torch.int16 if self.prec == "q14" else torch.complex64
        dt_out = torch.int32 if self.prec == "q14" else torch.complex64
        _need(surv, dt_in, "surv")
        _need(ref, dt_in, "ref")
        _need(out, dt_out, "out")
        L.check(self.lib.caf_exec_batched(self.handle, _ptr(surv), _ptr(ref), _ptr(out), _stream(surv.device)),
                "caf_exec_batched")
        return out

    def last_launches(self) -> int:
        c = ctypes.c_int32()
        L.check(self.lib.ndft_last_launches(self.handle, ctypes.byref(c)), "ndft_last_launches")
        return c.value

    def set_tuning(self, key: int, value: int):
        L.check(self.lib.ndft_set_tuning(self.handle, int(key), int(value)), "ndft_set_tuning")

    def nbytes(self) -> int:
        """Device bytes the plan holds (tables + workspace)."""
        b = ctypes.c_int64()
        L.check(self.lib.ndft_plan_bytes(self.handle, ctypes.byref(b)), "ndft_plan_bytes")
        return b.value

    def signature(self) -> str:
        return self._sig

    def query_error(self):
        L.check(self.lib.ndft_query_error(self.handle, _stream(self.device)), "ndft_query_error")

    def close(self):
        if getattr(self, "handle", None):
            L.check(self.lib.ndft_plan_destroy(self.handle), "ndft_plan_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def argmax(X: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    """Per-row index of the largest |X|^2 (lowest index on ties) and that value; X [rows, cols] complex64."""
    _need(X, torch.complex64, "X")
    X2 = X.reshape(X.shape[0], -1) if X.dim() > 1 else X.reshape(1, -1)
    rows, cols = X2.shape
    idx = torch.empty(rows, dtype=torch.int64, device=X.device)
    val = torch.empty(rows, dtype=torch.float32, device=X.device)
    L.check(L.load().ndft_argmax(_ptr(X2), rows, cols, _ptr(idx), _ptr(val), _stream(X.device)), "ndft_argmax")
    return idx, val


class CafFunction(torch.autograd.Function):
    """A = CAF(s_surv; s_ref) (Eq. 12a) with the hand-written adjoints as its backward.

    Gradient convention is PyTorch's for complex inputs: s_surv.grad = dL/dRe + j dL/dIm
    (s_ref likewise)."""

    @staticmethod
    def forward(ctx, s_surv, s_ref, plan: Plan, lag0: int, nlags: int):
        A = plan.caf(s_surv.detach().contiguous(), s_ref.detach().contiguous(), lag0, nlags)
        ctx.save_for_backward(s_surv, s_ref)
        ctx.plan, ctx.lag0, ctx.nlags = plan, lag0, nlags
        return A

    @staticmethod
    def backward(ctx, dA):
        s_surv, s_ref = ctx.saved_tensors
        ss, sr, g = s_surv.detach().contiguous(), s_ref.detach().contiguous(), dA.contiguous()
        want_surv, want_ref = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if want_ref:
            ds, dr = ctx.plan.caf_backward_inputs(ss, sr, ctx.lag0, ctx.nlags, g, surv=want_surv)
            return ds, dr, None, None, None
        if not want_surv:
            return None, None, None, None, None
        ds = ctx.plan.caf_backward(ss, sr, ctx.lag0, ctx.nlags, g)
        return ds, None, None, None, None


def caf_autograd(s_surv: torch.Tensor, s_ref: torch.Tensor, plan: Plan, lag0: int, nlags: int) -> torch.Tensor:
    return CafFunction.apply(s_surv, s_ref, plan, lag0, nlags)
