"""The C ABI without a GPU: the library builds for sm_103a, loads, and exports every entry
point that include/isycos.h declares; the binding's struct layouts match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(isycos_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_09131_gb300 import api
    return api.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_2204_09131_gb300 import api
    assert set(api.SIGNATURES) == _declared()


def test_struct_sizes_match_the_header():
    from paper_2204_09131_gb300 import api
    assert ctypes.sizeof(api.isycos_window) == 24
    assert ctypes.sizeof(api.isycos_mi_out) == 40
    assert ctypes.sizeof(api.isycos_result_window) == 32
    assert ctypes.sizeof(api.isycos_params) == 104
    assert ctypes.sizeof(api.isycos_stats) == 632
    assert ctypes.sizeof(api.isycos_tuning) == 400


def test_params_defaults_follow_the_paper(lib):
    from paper_2204_09131_gb300 import api
    p = api.isycos_params_default()
    # sigma = 0.2 on the normalised score; tau < 0 selects sigma / 4 (Sec. 8.3 settings)
    assert p.sigma == pytest.approx(0.2) and p.tau < 0
    assert p.k == 4 and p.score_kind == 0 and p.mode == 0 and p.pruning == 0


def test_create_fails_cleanly_without_a_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.isycos_create(ctypes.byref(h), 0, 0)
    assert st != 0 and not h.value
