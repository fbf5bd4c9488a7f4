"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every
function include/ndft.h declares, and rejects bad arguments before touching
the GPU.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_1402_0532_gb300 import _lib as L
from paper_1402_0532_gb300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ndft.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_lists_the_boundary():
    names = header_functions()
    for must in ("ndft_plan", "ndft_exec", "nfft_exec", "caf_exec", "caf_exec_batched", "caf_backward",
                 "caf_backward_inputs", "ndft_plan_destroy", "ndft_status_string", "ndft_query_error"):
        assert must in names
    assert sorted(L.EXPORTS) == names


def test_every_declared_symbol_is_exported(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_version(lib):
    assert lib.ndft_status_string(0) == b"ok"
    assert lib.ndft_status_string(L.E_INVALID) == b"invalid argument"
    assert lib.ndft_version() >= 100


def test_argument_errors_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.ndft_plan(ctypes.byref(h), None, None) == L.E_INVALID
    d = L.NdftDesc(n=0, max_batch=1)
    assert lib.ndft_plan(ctypes.byref(h), ctypes.byref(d), None) == L.E_INVALID
    d = L.NdftDesc(n=64, nbins=65, max_batch=1)
    assert lib.ndft_plan(ctypes.byref(h), ctypes.byref(d), None) == L.E_INVALID
    d = L.NdftDesc(n=64, max_batch=1, form=L.FORM_DIRECT, prec=L.PREC_BF16X2)
    assert lib.ndft_plan(ctypes.byref(h), ctypes.byref(d), None) == L.E_UNSUPPORTED
    d = L.NdftDesc(n=64, max_batch=1, flags=0x80)
    assert lib.ndft_plan(ctypes.byref(h), ctypes.byref(d), None) == L.E_INVALID
    assert lib.ndft_exec(None, None, None, 1, None) == L.E_INVALID
    assert lib.nfft_exec(None, None, None, 1, None) == L.E_INVALID
    assert lib.caf_exec(None, None, None, 0, 1, None, None) == L.E_INVALID
    assert lib.caf_exec_batched(None, None, None, None, None) == L.E_INVALID
    assert lib.caf_backward(None, None, None, 0, 1, None, None, None) == L.E_INVALID
    # no output at all, or no plan
    assert lib.caf_backward_inputs(None, None, None, 0, 1, None, None, None, None) == L.E_INVALID
    buf = ctypes.create_string_buffer(64)
    assert lib.caf_backward_inputs(None, None, None, 0, 1, None, None, ctypes.addressof(buf), None) == L.E_INVALID
    assert lib.ndft_argmax(None, -1, 4, None, None, None) == L.E_INVALID
    assert lib.ndft_argmax(None, 0, 4, None, None, None) == L.OK  # nothing to do
    assert lib.ndft_set_tuning(None, 0, 1) == L.E_INVALID
    assert lib.ndft_query_error(None, None) == L.E_INVALID
    assert lib.ndft_plan_destroy(None) == L.E_INVALID
    assert lib.ndft_plan_batched(ctypes.byref(h), None, 0, 0, 0, 0, None) == L.E_INVALID
    cpi = (L.NdftCpi * 1)(L.NdftCpi(n=0, nlags=1, nbins=1))
    assert lib.ndft_plan_batched(ctypes.byref(h), cpi, 1, 0, 0, 0, None) == L.E_INVALID
    # a lag window running past INT32_MAX is refused before any device call
    cpi = (L.NdftCpi * 1)(L.NdftCpi(n=1024, lag0=2**31 - 3, nlags=4, nbins=8))
    assert lib.ndft_plan_batched(ctypes.byref(h), cpi, 1, 0, 0, 0, None) == L.E_INVALID


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_1402_0532_gb300 import api
    with pytest.raises(TypeError):
        api._need(torch.zeros(4, dtype=torch.complex64), torch.complex64, "x")


def test_choose_form_crossover():
    """The form chooser: the plain form up to N = 64, the tensor-core form above
    (its measured crossover), each with its own precision."""
    pytest.importorskip("torch")
    from paper_1402_0532_gb300 import api
    assert api.choose_form(2) == ("direct", "fp32")
    assert api.choose_form(64) == ("direct", "fp32")
    assert api.choose_form(65) == ("ternary", "bf16x2")
    assert api.choose_form(65536) == ("ternary", "bf16x2")
