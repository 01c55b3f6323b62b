"""The C ABI library builds for sm_103a, loads, and exports every symbol include/*.h declares.

No compute calls: these run without a GPU.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(ot_assoc_\w+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ot_assoc_create", "ot_assoc_build_cost", "ot_assoc_solve", "ot_assoc_build_rates",
                 "ot_assoc_maxsinr", "ot_assoc_median_f32"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1805_01559_gb300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1805_01559_gb300 import binding
    assert _declared() <= set(binding.SIGNATURES), _declared() - set(binding.SIGNATURES)
    L = binding.lib()
    assert L.ot_assoc_version() >= 100
    assert L.ot_assoc_status_string(-4) == b"OT_ETIMEOUT"


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1805_01559_gb300 import binding
    L = binding.lib()
    h = ctypes.c_void_p()
    st = L.ot_assoc_create(ctypes.byref(h), 0, 0)
    assert st in (binding.OT_ECUDA, binding.OT_EINVAL)
    assert not h.value
