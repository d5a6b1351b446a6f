"""The C-ABI library loads and exports every entry point of include/ideq.h (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "ideq.h")


def header_functions():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ideq_[A-Za-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_19705_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert "ideq_solve" in names and "ideq_solve_backward" in names and len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared in ideq.h but not exported"


def test_binding_covers_header():
    from paper_2605_19705_gb300 import build
    build.build()
    from paper_2605_19705_gb300 import binding
    assert sorted(binding.EXPORTED) == header_functions()


def test_num_params_matches_synth_layout():
    from paper_2605_19705_gb300 import build
    build.build()
    from paper_2605_19705_gb300 import binding
    import numpy as np
    from synth import generators as G
    for widths in ([64, 128, 256, 512], [32, 64, 128, 256], [8, 16, 16, 32]):
        d = binding.net_desc({"type": "unet", "widths": widths, "n_rb": 2}, 3)
        n = binding.ideq_num_params(d)
        assert n == sum(int(np.prod(s)) for _, _, s, *_ in G.unet_layout(3, widths, 2))
    d = binding.net_desc({"type": "cnn", "chans": [1, 32, 32, 32, 1]}, 1)
    assert binding.ideq_num_params(d) == 19008


def test_null_context_calls_are_argument_errors(lib):
    """Context queries check their arguments before any CUDA call (no GPU needed)."""
    from paper_2605_19705_gb300 import binding
    lib.ideq_solve_graphed.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
    lib.ideq_launch_count.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
    lib.ideq_last_error.argtypes = [ctypes.c_void_p]
    lib.ideq_last_error.restype = ctypes.c_char_p
    g, n = ctypes.c_int(7), ctypes.c_int64(7)
    assert lib.ideq_solve_graphed(None, ctypes.byref(g)) == binding.IDEQ_ERR_ARG
    assert lib.ideq_launch_count(None, ctypes.byref(n)) == binding.IDEQ_ERR_ARG
    assert g.value == 7 and n.value == 7  # outputs untouched on error
    assert lib.ideq_last_error(None) == b"null context"
