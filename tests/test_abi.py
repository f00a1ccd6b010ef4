"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/fmm.h declares (no compute calls here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z0-9_]+)\s*\(", src)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_exports_declared_symbols():
    from paper_1108_5815_gb300 import build, fmm
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert "fmm_laplace3d" in declared and "fmm_direct" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(fmm.ABI_SYMBOLS) | {n for n in declared if n.startswith("fmm_")}
    for name in fmm.ABI_SYMBOLS:
        assert name in declared


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_1108_5815_gb300 import build, fmm
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    build.build()
    x = torch.zeros(4, 3)
    with pytest.raises(fmm.FmmError):
        fmm.laplace3d(x, torch.zeros(4), 4, 0.5, 8)
