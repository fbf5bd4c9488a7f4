"""The smoke check (one small invocation of every form against the
oracle) as part of the GPU suite, so it cannot break unnoticed."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_smoke():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    __graft_entry__.smoke()
