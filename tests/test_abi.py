"""CPU-side checks of the C ABI library: it builds, loads and exports every
function include/nufft_gb300.h declares (no GPU calls)."""
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
        with open(os.path.join(ROOT, "include", fn)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(nufft_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2102_08463_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "nufft_makeplan" in names and "nufft_execute" in names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_lists_every_symbol():
    from paper_2102_08463_gb300 import binding
    assert set(binding.EXPORTS) == _declared()


def test_strerror_and_default_opts_without_gpu(lib):
    from paper_2102_08463_gb300 import binding
    assert binding.strerror(-7) == "execute called before setpts"
    assert binding.strerror(12345) == "unknown error"
    o = binding.default_opts()
    assert o.method == 0 and o.upsampfac == 2.0 and o.msub == 0


def test_algorithmic_cost_per_point_matches_formulas():
    import bench
    # bytes per point at density 1 (fine grid = M cells): 2D 24/48, 3D 28/56
    for d, prec, want in ((2, 0, 24), (2, 1, 48), (3, 0, 28), (3, 1, 56)):
        W = dict(dim=d, prec=prec, M=1000, nf=[1000] + [1] * (d - 1))
        b, _ = bench.algorithmic_cost(W, 6, "spread")
        assert b == want * 1000
    # flops: 8 d w + (d+3) w^d per point -> 2D w=6: 276, 3D w=7: 2226
    _, f = bench.algorithmic_cost(dict(dim=2, prec=0, M=1, nf=[1, 1]), 6, "spread")
    assert f == 276
    _, f = bench.algorithmic_cost(dict(dim=3, prec=0, M=1, nf=[1, 1, 1]), 7, "spread")
    assert f == 2226
