"""The product path has no CPU fallback (CPU only).

Without a GPU every call that would compute fails with an error from the CUDA library, and
without the library nothing loads: nothing quietly computes on the host instead."""
import numpy as np
import pytest

from paper_1410_4054_gb300 import pk
from paper_1410_4054_gb300 import workloads as W


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


@pytest.mark.skipif(_has_gpu(), reason="checks the behaviour without a GPU")
def test_no_gpu_means_an_error_not_a_host_result():
    a = W.laplace_2d(8)
    with pytest.raises(pk.PkError) as e:
        pk.CSRMatrix(a.row_ptr, a.col, a.val)
    assert e.value.status == pk.PK_ERR_CUDA


def test_missing_library_fails_loudly(monkeypatch):
    def no_nvcc():
        raise RuntimeError("nvcc not found: the pk CUDA library cannot be built")

    monkeypatch.setattr(pk, "_lib", None)
    monkeypatch.setattr(pk._build, "build", no_nvcc)
    with pytest.raises(RuntimeError, match="cannot be built"):
        pk.lib()
    with pytest.raises(RuntimeError, match="cannot be built"):
        pk.csr_plan(np.array([0, 1], np.int32))
