"""The C-ABI library builds, loads, and exports every entry point that
include/*.h declares (the query API in ahpp.h, the measurement helpers in
ahpp_measure.h).

No kernel runs here: on a machine without a GPU the library must refuse
(AHPP_ECUDA), never fall back to the CPU.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_11606_gb300 import build
    build.build()
    from paper_2512_11606_gb300 import ahpp
    return ahpp.lib()


def header_functions():
    inc = os.path.join(ROOT, "include")
    names = set()
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(ahpp_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_2512_11606_gb300 import ahpp
    assert set(names) == set(ahpp.SIGNATURES), set(names) ^ set(ahpp.SIGNATURES)


def test_struct_sizes_match_header(lib):
    from paper_2512_11606_gb300 import ahpp
    # field lists mirror include/ahpp.h; sizes follow the C layout rules
    assert ctypes.sizeof(ahpp.Stats) == 4 * 4 + 8 * 2 + 8 * 7
    assert ctypes.sizeof(ahpp.GraphDesc) == 8 * 11
    c = ahpp.default_config()
    assert c.alpha == 0.15 and c.beta == 0.35 and c.algo == ahpp.AHPP_ASRP
    assert c.attr_bf16 == 1 and c.kahan == 1 and c.lambda_ == 0.0
    assert c.batch_chunk == 0


def test_no_cpu_fallback_without_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2512_11606_gb300 import ahpp, synth
    g = synth.make_graph(**synth.TINY)
    with pytest.raises(ahpp.AhppError) as ei:
        ahpp.Graph.from_arrays(g)
    assert ei.value.code == ahpp.AHPP_ECUDA
    assert "no CUDA device" in str(ei.value)


def test_last_error_is_empty_string_initially(lib):
    assert isinstance(lib.ahpp_last_error(), bytes)
