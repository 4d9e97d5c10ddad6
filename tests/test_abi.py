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


def _c_struct(name):
    """(field, C type, array length) of typedef struct { ... } name; in the header."""
    with open(os.path.join(ROOT, "include", "nufft_gb300.h")) as fh:
        text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    out = []
    for decl in body.split(";"):
        m = re.match(r"\s*([a-z_ ]+?)\s*(\*?)\s*([a-z_0-9]+)\s*(?:\[(\d+)\])?\s*$", decl)
        if m:
            out.append((m.group(3), m.group(1) + m.group(2), int(m.group(4) or 1)))
    return out


@pytest.mark.parametrize("c_name,py_name", [("nufft_opts", "Opts"),
                                            ("nufft_tune_trial", "TuneTrial")])
def test_ctypes_structs_mirror_the_header(c_name, py_name):
    from paper_2102_08463_gb300 import binding
    ctype = {"int": ctypes.c_int, "double": ctypes.c_double, "void*": ctypes.c_void_p}
    fields = _c_struct(c_name)
    py = getattr(binding, py_name)._fields_
    assert [f[0] for f in fields] == [f[0] for f in py]
    for (name, ct, n), (_, pt) in zip(fields, py):
        want = ctype[ct] * n if n > 1 else ctype[ct]
        assert ctypes.sizeof(pt) == ctypes.sizeof(want) and \
            getattr(pt, "_type_", pt) == getattr(want, "_type_", want), name


def test_default_opts_fill_every_field(lib):
    from paper_2102_08463_gb300 import binding
    o = binding.Opts()
    ctypes.memset(ctypes.byref(o), 0x5a, ctypes.sizeof(o))
    lib.nufft_default_opts(ctypes.byref(o))
    assert o.method == 0 and list(o.bin) == [0, 0, 0] and o.msub == 0
    assert o.upsampfac == 2.0 and not o.stream and o.threads == 0 and o.ctas_per_sm == 0
    assert o.use_picker == 0 and o.unordered_bins == 0 and o.debug_checks == 0


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


def test_picker_features_without_gpu(lib):
    from paper_2102_08463_gb300 import binding as nb
    # 2D type 1, N = 1024^2, eps 1e-5: w = 6, n = 2048^2; M = n_tot; default tiles (SM,
    # (16 - w) x 16 = 10 x 16 bins, M_sub 1024, 256 threads)
    import math
    f = nb.picker_features(1, (1024, 1024), 1e-5, 2048 * 2048, 1.5, "sm")
    want = [0, 0, 0, 6 / 16, 22 / 32, 0.0, 1.5 / 16, 1, 0, math.log2(160) / 12, 10 / 12, 1.0]
    assert f == pytest.approx(want, abs=1e-7)
    # 3D type 2 double, N = 100^3 at eps 1e-9 (w = 10, n = 200^3), GM, 8x8x4 bins
    f = nb.picker_features(2, (100, 100, 100), 1e-9, 1000, 0.0, "gm", bins=(8, 8, 4), msub=256,
                           threads=128)
    assert f[:4] == pytest.approx([1, 1, 1, 10 / 16])
    assert f[4] == pytest.approx(math.log2(200 ** 3) / 32, abs=1e-7)
    assert f[5] == pytest.approx(math.log2(1000 / 200 ** 3) / 8, abs=1e-7)
    assert f[6:] == pytest.approx([0, 0, 1, 8 / 12, 8 / 12, 0.5], abs=1e-7)
    with pytest.raises(nb.NufftError):
        nb.picker_features(1, (64, 64), 1e-5, 100, 0.0, "auto")
    with pytest.raises(nb.NufftError):
        nb.picker_features(1, (64, 64), 1e-9, 100, 0.0, "sm", prec=0)


def test_sigma_candidates_and_pick_without_gpu(lib):
    import math
    from paper_2102_08463_gb300 import binding as nb
    from paper_2102_08463_gb300 import picker
    lib = nb.load()
    # sigma = 1.25 at eps 1e-3: w = ceil(3 / 0.6) + 1 = 6, n = next235(1.25 * 1024) = 1280
    f = nb.picker_features(1, (1024, 1024), 1e-3, 1280 * 1280, 0.0, "sm", upsampfac=1.25)
    assert f[3] == pytest.approx(6 / 16)
    assert f[4] == pytest.approx(math.log2(1280 * 1280) / 32, abs=1e-7)
    assert f[5] == pytest.approx(0.0, abs=1e-7)
    # the sigma = 1.25 plan exists in single precision for eps >= 1e-4 only, and in
    # double precision while w <= 16 (w = ceil(log10(1/eps) / 0.6) + 1)
    assert picker.sigma125_width(1, (64, 64), 1e-3, 100, 0) == 6
    assert picker.sigma125_width(1, (64, 64), 1e-5, 100, 0) is None
    assert picker.sigma125_width(2, (64, 64, 64), 1e-9, 100, 1) == 16
    assert picker.sigma125_width(2, (64, 64), 1e-11, 100, 1) is None
    assert picker.trial_sigma([3, 8, 8, 1, 256, 128, 1.0]) == 2.0
    assert picker.trial_sigma([3, 8, 8, 1, 256, 128, 1.25, 1.0]) == 1.25
    # nufft_pick: argument errors and an eps no sigma reaches leave opts as given,
    # and with no picker installed the answer is sigma = 2 with automatic tiles --
    # none of these touch the device
    arr = (ctypes.c_int64 * 3)(64, 64, 1)
    o = nb.default_opts()
    o.msub = 77
    assert lib.nufft_pick(4, 2, arr, 1e-3, 0, 0, None, None, None, None, ctypes.byref(o)) \
        == nb.NUFFT_ERR_ARG
    assert lib.nufft_pick(1, 2, arr, 1e-3, -1, 0, None, None, None, None, ctypes.byref(o)) \
        == nb.NUFFT_ERR_ARG
    assert lib.nufft_pick(1, 2, arr, 1e-3, 0, 5, None, None, None, None, ctypes.byref(o)) \
        == nb.NUFFT_ERR_ARG
    assert lib.nufft_pick(1, 2, arr, 1e-7, 0, 0, None, None, None, None, ctypes.byref(o)) \
        == nb.NUFFT_ERR_EPS
    assert o.msub == 77
    nb.Picker.uninstall()
    assert lib.nufft_pick(1, 2, arr, 1e-3, 0, 0, None, None, None, None, ctypes.byref(o)) == 0
    assert (o.upsampfac, o.method, tuple(o.bin), o.msub, o.threads) == (2.0, 0, (0, 0, 0), 0, 0)
    assert lib.nufft_pick(2, 2, arr, 1e-11, 1, 0, None, None, None, None, ctypes.byref(o)) == 0
    assert o.upsampfac == 2.0
