"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself or with the GPU library: each
check uses a closed form, a library routine (numpy FFT, numpy sort, scipy
quadrature), an invariant, or a value printed in the paper (tests/golden/).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2102_08463_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pts(dim, M, seed, kind="rand"):
    return wl.points(kind, dim, M, seed, dtype=np.float64)


# ---------------------------------------------------------------------------
# Parameters (Sec. 3)
# ---------------------------------------------------------------------------
def test_kernel_width_matches_paper_examples():
    with open(os.path.join(GOLDEN, "params_sec3.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    assert rows
    for r in rows:
        eps, wmin, wmax = float(r[0]), int(r[1]), int(r[2])
        w = oracle.kernel_width(eps)
        assert wmin <= w <= wmax, (eps, w)


def test_kernel_width_monotone_and_beta_rule():
    ws = [oracle.kernel_width(10.0 ** -e) for e in np.linspace(1, 14, 131)]
    assert all(a <= b for a, b in zip(ws, ws[1:]))
    # beta = 2.30 w (Sec. 3); w grows by exactly one per decade of tolerance
    assert oracle.kernel_width(1e-3) - oracle.kernel_width(1e-2) == 1
    assert oracle.kernel_beta(6) == pytest.approx(13.8)


def test_next235_brute_force():
    def smooth(v):
        for p in (2, 3, 5):
            while v % p == 0:
                v //= p
        return v == 1
    for n in range(1, 600):
        m = oracle.next235(n)
        assert m >= n and smooth(m)
        assert not any(smooth(v) for v in range(n, m))
    # fine grids of the paper's test sizes, sigma = 2 (Sec. 5.3: N = 1000^2, 100^3)
    assert oracle.fine_grid_size(1000, 6) == 2000
    assert oracle.fine_grid_size(100, 6) == 200
    assert oracle.fine_grid_size(4, 13) == 27   # max(2N, 2w) = 26 -> 27 = 3^3


# ---------------------------------------------------------------------------
# ES kernel and its Fourier transform
# ---------------------------------------------------------------------------
def test_es_kernel_special_values():
    beta = 13.8
    assert oracle.es_kernel(np.array([0.0]), beta)[0] == 1.0
    assert oracle.es_kernel(np.array([1.0]), beta)[0] == pytest.approx(math.exp(-beta), rel=1e-15)
    assert oracle.es_kernel(np.array([-1.0000001, 1.5]), beta).tolist() == [0.0, 0.0]
    lib = oracle._load()
    for z in (-0.7, 0.0, 0.3, 0.99):
        assert lib.orc_es_kernel(z, beta) == pytest.approx(oracle.es_kernel(np.array([z]), beta)[0], rel=1e-15)


def test_phihat_beta_zero_closed_form():
    # beta = 0 makes phi the indicator of [-1, 1]: phihat(xi) = 2 sin(xi) / xi
    xi = np.linspace(0.1, 12.0, 37)
    assert np.allclose(oracle.phihat(xi, 0.0), 2 * np.sin(xi) / xi, rtol=0, atol=1e-13)


def test_phihat_node_doubling_and_scipy_quad():
    from scipy.integrate import quad
    for w in (3, 6, 10, 13, 16):
        beta = oracle.kernel_beta(w)
        xi = np.linspace(0.0, w * math.pi / 2.0, 9)
        a = oracle.phihat(xi, beta, 200)
        b = oracle.phihat(xi, beta, 400)
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))
        for v in xi[::4]:
            ref, _ = quad(lambda z: math.exp(beta * (math.sqrt(1 - z * z) - 1)) * math.cos(v * z),
                          -1, 1, epsabs=1e-15, epsrel=1e-13, limit=400)
            assert oracle.phihat(np.array([v]), beta)[0] == pytest.approx(ref, rel=1e-11, abs=1e-15)


# ---------------------------------------------------------------------------
# O1: exact sums
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("iflag", [+1, -1])
def test_direct_type1_on_grid_points_is_a_dft(iflag):
    # points on the N-grid x = -pi + 2 pi j / N turn Eq. (2d1) into a plain DFT:
    # f_k = (-1)^{k1+k2} sum_j c_j e^{iflag 2 pi i (k.j)/N}
    N1, N2 = 6, 5
    j1, j2 = np.meshgrid(np.arange(N1), np.arange(N2), indexing="xy")
    x = -math.pi + 2 * math.pi * j1.ravel() / N1
    y = -math.pi + 2 * math.pi * j2.ravel() / N2
    rng = np.random.default_rng(3)
    cg = rng.standard_normal((N2, N1)) + 1j * rng.standard_normal((N2, N1))
    f = oracle.direct_type1([x, y], cg.ravel(), (N1, N2), iflag)
    full = np.fft.ifft2(cg) * (N1 * N2) if iflag > 0 else np.fft.fft2(cg)
    k1 = oracle.modes_1d(N1)
    k2 = oracle.modes_1d(N2)
    ref = full[np.ix_(k2 % N2, k1 % N1)] * ((-1.0) ** (k2[:, None] + k1[None, :]))
    assert np.max(np.abs(f - ref)) < 1e-12


def test_direct_type2_on_grid_points_is_a_dft():
    N1, N2, N3 = 4, 3, 5
    J = np.meshgrid(np.arange(N1), np.arange(N2), np.arange(N3), indexing="ij")
    x, y, z = (-math.pi + 2 * math.pi * J[i].transpose(2, 1, 0).ravel() / n
               for i, n in enumerate((N1, N2, N3)))
    rng = np.random.default_rng(4)
    f = rng.standard_normal((N3, N2, N1)) + 1j * rng.standard_normal((N3, N2, N1))
    c = oracle.direct_type2([x, y, z], f, iflag=+1)      # exponent -i k.x
    k = [oracle.modes_1d(n) for n in (N1, N2, N3)]
    sgn = (-1.0) ** (k[2][:, None, None] + k[1][None, :, None] + k[0][None, None, :])
    g = np.zeros((N3, N2, N1), dtype=complex)
    g[np.ix_(k[2] % N3, k[1] % N2, k[0] % N1)] = f * sgn
    ref = np.fft.fftn(g)
    assert np.max(np.abs(c - ref.ravel())) < 1e-12


def test_direct_sign_closed_form():
    # a unit mass at x = (pi/2, 0): f_{(1,0)} = e^{i pi/2} = i for iflag = +1, -i for -1
    for iflag, want in ((+1, 1j), (-1, -1j)):
        f = oracle.direct_type1([np.array([math.pi / 2]), np.array([0.0])], np.array([1.0 + 0j]),
                                (4, 4), iflag)
        assert abs(f[2, 3] - want) < 1e-15          # (k2, k1) = (0, 1)
        assert abs(f[2, 0] - (-1.0)) < 1e-15      # k1 = -2: e^{-+ i pi} = -1


def test_direct_adjoint_shift_and_conjugate_symmetry():
    M, N = 60, (7, 6)
    pts = _pts(2, M, 11)
    c = wl.strengths(M, 12, np.complex128)
    f = wl.modes(N, 13, np.complex128)
    a1 = oracle.direct_type1(pts, c, N, +1)
    a2 = oracle.direct_type2(pts, f, +1)
    lhs = np.vdot(f.ravel(), a1.ravel())
    rhs = np.vdot(a2, c)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # shift: x -> x + delta multiplies f_k by e^{i k . delta}
    d = (0.3, -0.2)
    a1s = oracle.direct_type1([pts[0] + d[0], pts[1] + d[1]], c, N, +1)
    k1 = oracle.modes_1d(N[0])
    k2 = oracle.modes_1d(N[1])
    ph = np.exp(1j * (k1[None, :] * d[0] + k2[:, None] * d[1]))
    assert np.max(np.abs(a1s - a1 * ph)) < 1e-12 * np.max(np.abs(a1))
    # real strengths: f_{-k} = conj(f_k) on the symmetric part of I_N
    fr = oracle.direct_type1(pts, c.real.astype(complex), (7, 7), +1)
    assert np.max(np.abs(fr - np.conj(fr[::-1, ::-1]))) < 1e-12


def test_direct_sampled_modes_and_targets_match_full():
    M, N = 40, (5, 4, 3)
    pts = _pts(3, M, 21)
    c = wl.strengths(M, 22, np.complex128)
    full = oracle.direct_type1(pts, c, N).ravel()
    idx = np.array([0, 7, 33, 59])
    assert np.array_equal(oracle.direct_type1(pts, c, N, modes=idx), full[idx])
    f = wl.modes(N, 23, np.complex128)
    full2 = oracle.direct_type2(pts, f)
    tg = np.array([1, 5, 39])
    assert np.array_equal(oracle.direct_type2(pts, f, targets=tg), full2[tg])


# ---------------------------------------------------------------------------
# O2: the three-step algorithm, pinned to O1
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,iflag", [(2, +1), (2, -1), (3, +1)])
def test_pipeline_tight_matches_direct(dim, iflag):
    N = (12, 10) if dim == 2 else (8, 6, 7)
    M = 150
    pts = _pts(dim, M, 31 + dim)
    c = wl.strengths(M, 32, np.complex128)
    f = wl.modes(N, 33, np.complex128)
    t1 = oracle.nufft_type1(pts, c, N, eps=1e-14, iflag=iflag)
    d1 = oracle.direct_type1(pts, c, N, iflag)
    assert oracle.rel_l2(t1, d1) < 1e-13
    t2 = oracle.nufft_type2(pts, f, eps=1e-14, iflag=iflag)
    d2 = oracle.direct_type2(pts, f, iflag)
    assert oracle.rel_l2(t2, d2) < 1e-13


@pytest.mark.parametrize("eps", [1e-2, 1e-5, 1e-9, 1e-12])
def test_pipeline_error_close_to_eps(eps):
    # Sec. 3: the width rule "typically gives relative l2 errors close to eps".
    # Measured with the exact sums, the rule lands between 1x and 3x eps in 2D
    # (up to ~4x in 3D at eps <= 1e-9); "close" is read as within 5x, and a
    # kernel much wider than the rule asks for would show up as far below eps.
    N, M = (32, 30), 2000
    pts = _pts(2, M, 41)
    c = wl.strengths(M, 42, np.complex128)
    e1 = oracle.rel_l2(oracle.nufft_type1(pts, c, N, eps), oracle.direct_type1(pts, c, N))
    assert eps / 1000 < e1 < 5 * eps
    f = wl.modes(N, 43, np.complex128)
    e2 = oracle.rel_l2(oracle.nufft_type2(pts, f, eps), oracle.direct_type2(pts, f))
    assert eps / 1000 < e2 < 5 * eps


def test_pipeline_adjoint_to_rounding():
    # with a fixed w-cell window, approximate type 2 is the exact adjoint of type 1
    N, M = (16, 12, 10), 300
    pts = _pts(3, M, 51)
    c = wl.strengths(M, 52, np.complex128)
    f = wl.modes(N, 53, np.complex128)
    a = oracle.nufft_type1(pts, c, N, eps=1e-3)
    b = oracle.nufft_type2(pts, f, eps=1e-3)
    lhs = np.vdot(f.ravel(), a.ravel())
    rhs = np.vdot(b, c)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_spread_interp_transpose_and_mass():
    n = (20, 18)
    w, beta = 5, oracle.kernel_beta(5)
    M = 70
    pts = _pts(2, M, 61)
    c = wl.strengths(M, 62, np.complex128)
    b = wl.modes(n, 63, np.complex128)
    s = oracle.spread(pts, c, n, w, beta)
    i = oracle.interp(pts, b, w, beta)
    assert abs(np.vdot(b.ravel(), s.ravel()) - np.vdot(i, c)) < 1e-12 * np.abs(c).sum()
    # Poisson summation: sum_l psi(l h - x) = psihat(0)/h up to O(eps) aliasing
    mass = s.sum()
    per_axis = oracle.phihat(np.array([0.0]), beta)[0] * w / 2.0
    assert abs(mass - c.sum() * per_axis ** 2) < 1e-3 * abs(c.sum()) * per_axis ** 2
    # periodicity: moving every point by 2 pi leaves the grid unchanged
    s2 = oracle.spread([pts[0] + 2 * math.pi, pts[1] - 2 * math.pi], c, n, w, beta)
    assert np.max(np.abs(s2 - s)) < 1e-12


def test_planted_sign_mistake_is_caught(monkeypatch):
    # dropping the (-1)^k grid-origin factor must break O2 vs O1
    N, M = (10, 8), 100
    pts = _pts(2, M, 71)
    c = wl.strengths(M, 72, np.complex128)
    good = oracle.nufft_type1(pts, c, N, eps=1e-10)
    ref = oracle.direct_type1(pts, c, N)
    assert oracle.rel_l2(good, ref) < 1e-9
    orig = oracle.correction_1d
    monkeypatch.setattr(oracle, "correction_1d", lambda *a, **k: np.abs(orig(*a, **k)))
    bad = oracle.nufft_type1(pts, c, N, eps=1e-10)
    assert oracle.rel_l2(bad, ref) > 0.1


# ---------------------------------------------------------------------------
# O3: bin-sort
# ---------------------------------------------------------------------------
_PI40 = Fraction("3.1415926535897932384626433832795028841971")


def test_cells_contain_the_point_exactly():
    # l must satisfy l <= (x+pi) n / (2 pi) < l+1 (mod n) in exact arithmetic
    x = np.concatenate([wl.points("rand", 1, 3000, 81, np.float32)[0].astype(np.float64),
                        np.array([-math.pi, math.pi, float(np.float32(math.pi)),
                                  float(np.float32(-math.pi)), 0.0, -0.0, 3 * math.pi - 1e-9,
                                  -3 * math.pi, 1e-30, -1e-30, 2.5, -2.5])])
    for n in (16, 27, 2048, 250):
        cell, frac = oracle.cells(x, n)
        assert cell.min() >= 0 and cell.max() < n
        for xv, l, fr in zip(x, cell, frac):
            u = (Fraction(float(xv)) + _PI40) * n / (2 * _PI40)
            u = u - n * math.floor(u / n)
            if abs(u - round(u)) < Fraction(1, 10 ** 9):
                continue          # within rounding of a cell boundary: either side is fine
            assert math.floor(u) == l
            assert abs(float(u - l) - fr) < 1e-12


def test_binsort_is_the_stable_sort_by_bin():
    n, m = (40, 36, 20), (16, 16, 2)
    M = 4000
    for kind in ("rand", "cluster"):
        pts = wl.points(kind, 3, M, 91, np.float32, n=n)
        pts = [p.astype(np.float64) for p in pts]
        binidx, counts, t = oracle.binsort(pts, n, m)
        # bin from the cells, x fastest (Sec. 4.1)
        nb = [(a + b - 1) // b for a, b in zip(n, m)]
        cl = [oracle.cells(p, ni)[0] for p, ni in zip(pts, n)]
        want = cl[0] // m[0] + nb[0] * (cl[1] // m[1] + nb[1] * (cl[2] // m[2]))
        assert np.array_equal(binidx, want)
        assert np.array_equal(t, np.argsort(binidx, kind="stable"))
        assert np.array_equal(counts, np.bincount(binidx, minlength=int(np.prod(nb))))


def test_subproblems_cover_each_bin():
    counts = np.array([0, 5, 1024, 1025, 3000, 1])
    rows = oracle.subproblems(counts, 1024)
    assert rows[:, 2].max() <= 1024
    for b, cnt in enumerate(counts):
        assert rows[rows[:, 0] == b, 2].sum() == cnt
    assert np.array_equal(rows[:, 1], np.concatenate([[0], np.cumsum(rows[:, 2])[:-1]]))


# ---------------------------------------------------------------------------
# sigma = 1.25 (not in the paper; the width / shape reading is checked here
# against the exact sums, which are pinned above)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6, 1e-8])
def test_sigma125_width_rule_meets_eps(eps):
    N, M = (40, 36), 3000
    pts = _pts(2, M, 41)
    c = wl.strengths(M, 42, np.complex128)
    exact = oracle.direct_type1(pts, c, N)
    w = oracle.kernel_width(eps, 1.25)
    e_w = oracle.rel_l2(oracle.nufft_type1(pts, c, N, w=w, sigma=1.25), exact)
    e_w1 = oracle.rel_l2(oracle.nufft_type1(pts, c, N, w=w - 1, sigma=1.25), exact)
    assert e_w <= eps            # the calibrated width reaches the tolerance
    assert e_w1 > e_w            # one cell narrower is measurably worse
    assert oracle.Params(N, eps, 1.25).n == (50, 45)   # 2^a 3^b 5^c >= 1.25 N


# ---------------------------------------------------------------------------
# 1D (the d = 1 case of Eq. 2d1 / 2d2 and of the algorithm of Sec. 3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("iflag", [+1, -1])
def test_direct_1d_on_grid_points_is_a_dft(iflag):
    N = 9
    x = -math.pi + 2 * math.pi * np.arange(N) / N
    rng = np.random.default_rng(81)
    c = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    f = oracle.direct_type1([x], c, (N,), iflag)
    full = np.fft.ifft(c) * N if iflag > 0 else np.fft.fft(c)
    k = oracle.modes_1d(N)
    assert np.max(np.abs(f - full[k % N] * (-1.0) ** k)) < 1e-12
    fm = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    g = np.zeros(N, dtype=complex)
    g[k % N] = fm * (-1.0) ** k
    ref = np.fft.fft(g) if iflag > 0 else np.fft.ifft(g) * N
    assert np.max(np.abs(oracle.direct_type2([x], fm, iflag) - ref)) < 1e-12


@pytest.mark.parametrize("iflag", [+1, -1])
def test_pipeline_1d_tight_matches_direct(iflag):
    N, M = (33,), 400
    pts = _pts(1, M, 82)
    c = wl.strengths(M, 83, np.complex128)
    f = wl.modes(N, 84, np.complex128)
    assert oracle.rel_l2(oracle.nufft_type1(pts, c, N, eps=1e-14, iflag=iflag),
                         oracle.direct_type1(pts, c, N, iflag)) < 1e-13
    assert oracle.rel_l2(oracle.nufft_type2(pts, f, eps=1e-14, iflag=iflag),
                         oracle.direct_type2(pts, f, iflag)) < 1e-13


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-10])
def test_pipeline_1d_error_close_to_eps(eps):
    N, M = (200,), 3000
    pts = _pts(1, M, 85)
    c = wl.strengths(M, 86, np.complex128)
    e1 = oracle.rel_l2(oracle.nufft_type1(pts, c, N, eps), oracle.direct_type1(pts, c, N))
    assert eps / 1000 < e1 < 5 * eps
    f = wl.modes(N, 87, np.complex128)
    e2 = oracle.rel_l2(oracle.nufft_type2(pts, f, eps), oracle.direct_type2(pts, f))
    assert eps / 1000 < e2 < 5 * eps


def test_spread_interp_1d_transpose_mass_periodicity():
    n, w = (40,), 7
    beta = oracle.kernel_beta(w)
    M = 90
    pts = _pts(1, M, 88)
    c = wl.strengths(M, 89, np.complex128)
    b = wl.modes(n, 90, np.complex128)
    s = oracle.spread(pts, c, n, w, beta)
    i = oracle.interp(pts, b, w, beta)
    assert abs(np.vdot(b, s) - np.vdot(i, c)) < 1e-12 * np.abs(c).sum()
    per_axis = oracle.phihat(np.array([0.0]), beta)[0] * w / 2.0
    assert abs(s.sum() - c.sum() * per_axis) < 1e-5 * abs(c.sum()) * per_axis
    s2 = oracle.spread([pts[0] - 4 * math.pi], c, n, w, beta)
    assert np.max(np.abs(s2 - s)) < 1e-12
    # a single point: its w weights, one per cell of its window, and nothing else
    one = oracle.spread([np.array([0.1])], np.array([1.0 + 0j]), n, w, beta)
    assert np.count_nonzero(one) == w


# ---------------------------------------------------------------------------
# type 3 exact sum (nonuniform frequencies)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_direct_type3_brute_force_and_integer_frequencies(dim):
    M, K = 23, 17
    pts = _pts(dim, M, 91 + dim)
    c = wl.strengths(M, 92, np.complex128)
    rng = np.random.default_rng(93)
    s = [rng.uniform(-20, 20, K) for _ in range(dim)]
    f = oracle.direct_type3(pts, c, s, +1)
    phase = sum(np.multiply.outer(s[d], pts[d]) for d in range(dim))
    ref = np.exp(1j * phase) @ c
    assert np.max(np.abs(f - ref)) < 1e-11 * np.abs(c).sum()
    assert np.max(np.abs(oracle.direct_type3(pts, c, s, -1) - np.exp(-1j * phase) @ c)) \
        < 1e-11 * np.abs(c).sum()
    # at the integer frequencies of I_N it is the type 1 sum
    N = (5, 4, 3)[:dim]
    k = np.meshgrid(*[oracle.modes_1d(n) for n in reversed(N)], indexing="ij")
    kk = [k[dim - 1 - d].ravel().astype(float) for d in range(dim)]
    f1 = oracle.direct_type1(pts, c, N, +1).ravel()
    assert np.max(np.abs(oracle.direct_type3(pts, c, kk, +1) - f1)) < 1e-13 * np.abs(c).sum()


def test_direct_type3_shift_is_a_modulation():
    # s -> s + d multiplies each term by e^{i d.x_j}: type 3 at s + d is type 3 at s
    # of the modulated strengths c_j e^{i d.x_j}
    M, K = 40, 11
    pts = _pts(2, M, 94)
    c = wl.strengths(M, 95, np.complex128)
    rng = np.random.default_rng(96)
    s = [rng.uniform(-50, 50, K), rng.uniform(-50, 50, K)]
    d = (0.37, -1.9)
    a = oracle.direct_type3(pts, c, [s[0] + d[0], s[1] + d[1]])
    cm = c * np.exp(1j * (d[0] * pts[0] + d[1] * pts[1]))
    b = oracle.direct_type3(pts, cm, s)
    assert np.max(np.abs(a - b)) < 1e-12 * np.abs(c).sum()
