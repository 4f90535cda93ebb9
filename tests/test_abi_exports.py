"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/rorbk.h declares (no device work: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "rorbk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rorbk_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["rorbk_setup", "rorbk_solve", "rorbk_free"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2510_02156_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2510_02156_gb300 import binding
    assert sorted(binding.SIGNATURES) == declared_symbols()


def test_binding_raises_without_device():
    """With no CUDA device the setup call must fail loudly, not fall back."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    from paper_2510_02156_gb300 import binding
    with pytest.raises(Exception):
        binding.Handle(np.array([0, 1]), np.array([0]), np.array([1.0]), 1, 1, 1, 0.0,
                       stream=0)
