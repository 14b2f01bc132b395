"""The C ABI library builds for sm_103a, loads, and exports every function
declared in include/sam.h; the binding declares exactly those names; the
oracle and the CUDA sources share no code.  CPU only (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    text = open(os.path.join(ROOT, "include", "sam.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sam_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_17656_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _header_functions()
    for required in ("sam_create", "sam_destroy", "sam_pattern_build", "sam_build", "sam_build_batched",
                     "sam_residual", "sam_apply", "sam_build_backward", "sam_tune", "sam_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header():
    from paper_2406_17656_gb300 import sam

    assert sorted(sam.exported_symbols()) == _header_functions()


def test_library_is_built_for_sm103a(lib):
    from paper_2406_17656_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_oracle_and_cuda_path_share_no_code():
    csrc = glob.glob(os.path.join(ROOT, "paper_2406_17656_gb300", "csrc", "*"))
    for f in csrc:
        assert "oracle" not in open(f).read().lower().replace("oracle-free", ""), f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.c")) + glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        src = open(f).read()
        assert "paper_2406_17656_gb300" not in src and "csrc" not in src, f
    pkg = glob.glob(os.path.join(ROOT, "paper_2406_17656_gb300", "*.py"))
    for f in pkg:
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src, f


def test_binding_fails_loudly_without_a_gpu():
    import torch

    from paper_2406_17656_gb300 import sam

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        sam.Handle()
