"""FP64 CPU oracle for the 1D/2D/3D type 1 and type 2 NUFFT of arXiv 2102.08463
(and the exact type 3 sum).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the GPU library never
does, and this package never imports the GPU library.

Two parts, as the paper's own accuracy study does (Sec. 5.3 measures errors
against a tight-tolerance CPU reference):

* O1 -- exact sums, Eq. (2d1) and Eq. (2d2), in FP64 with compensated phases and
  compensated summation (``direct_type1`` / ``direct_type2``); optionally only a
  sampled subset of modes or targets.  ``direct_type3`` is the same sum at real
  (nonuniform) frequencies: the type 3 transform, which the paper defines by
  reference only and lists as future work, so its oracle is the definition.
  1D is the d = 1 case of every sum and of the three-step algorithm (the paper
  gives the method per dimension, Sec. 3; 1D is also listed as future work).
* O2 -- the plain three-step algorithm of Sec. 3.1 / 3.2 in FP64
  (``nufft_type1`` / ``nufft_type2``): C spreading / interpolation loops,
  ``numpy.fft`` as the FFT step, and the deconvolution factors of Sec. 3.1 step 3
  from a Gauss-Legendre quadrature of the ES kernel's Fourier transform.
* O3 -- the bin-sort of Sec. 4.1 (``binsort``), a stable counting sort.

Parameter rules follow Sec. 3: w = ceil(log10(1/eps)) + 1, beta = 2.30 w,
n_i = smallest 2^a 3^b 5^c >= max(sigma N_i, 2w), sigma = 2.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "nufft_oracle.c")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-std=gnu11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.orc_es_kernel.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_es_kernel.restype = ctypes.c_double
        lib.orc_direct_type1.argtypes = [ctypes.c_int, I64, P, P, P, P, ctypes.c_int,
                                         P, I64, P, P]
        lib.orc_direct_type2.argtypes = [ctypes.c_int, I64, P, P, P, P, ctypes.c_int,
                                         P, I64, P, P]
        lib.orc_direct_type3.argtypes = [ctypes.c_int, I64, P, P, P, P, ctypes.c_int,
                                         I64, P, P, P, P]
        lib.orc_spread.argtypes = [ctypes.c_int, I64, P, P, P, P, P, ctypes.c_int,
                                   ctypes.c_double, P]
        lib.orc_interp.argtypes = [ctypes.c_int, I64, P, P, P, P, P, ctypes.c_int,
                                   ctypes.c_double, P]
        lib.orc_cells.argtypes = [I64, P, I64, P, P]
        lib.orc_binsort.argtypes = [ctypes.c_int, I64, P, P, P, P, P, P, P, P]
        lib.orc_binsort.restype = I64
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


# ---------------------------------------------------------------------------
# Parameters, Sec. 3
# ---------------------------------------------------------------------------
def kernel_width(eps: float, sigma: float = 2.0) -> int:
    """Number of fine-grid cells w that one point's kernel covers per axis.

    sigma = 2: w = ceil(log10(1/eps)) + 1 (Sec. 3).  Powers of ten map to their
    nominal width (a 1e-10 relative guard absorbs the rounding of 1/eps), so
    1e-2 -> 3, 1e-5 -> 6, 1e-6 -> 7, 1e-9 -> 10, 1e-12 -> 13.  Clamped to [2, 16].
    sigma = 1.25 (not in the paper): w = ceil(log10(1/eps) / 0.6) + 1, the
    width calibrated against this oracle (see the sigma = 1.25 tests).
    """
    if not (eps > 0):
        raise ValueError("eps must be positive")
    digits = -math.log10(eps)
    if sigma == 2.0:
        w = math.ceil(digits - 1e-10) + 1
    elif sigma == 1.25:
        w = math.ceil(digits / 0.6 - 1e-10) + 1
    else:
        raise ValueError("sigma must be 2 or 1.25")
    return int(min(max(w, 2), 16))


def kernel_beta(w: int, sigma: float = 2.0) -> float:
    """ES shape parameter: beta = 2.30 w for sigma = 2 (Sec. 3).

    For sigma = 1.25 the same cutoff argument is scaled: beta is proportional
    to the distance (1 - 1/(2 sigma)) between the retained band edge and the
    first alias, so beta = 2.30 w (1 - 1/(2 sigma)) / (1 - 1/4).
    """
    if sigma == 2.0:
        return 2.30 * w
    return 2.30 * w * (1.0 - 1.0 / (2.0 * sigma)) / 0.75


def next235(n: int) -> int:
    """Smallest integer >= n of the form 2^a 3^b 5^c (Sec. 3)."""
    n = max(int(n), 1)
    while True:
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            return n
        n += 1


def fine_grid_size(N: int, w: int, sigma: float = 2.0) -> int:
    """n_i = smallest 2^a 3^b 5^c >= max(sigma N_i, 2w) (Sec. 3)."""
    return next235(max(int(math.ceil(sigma * N - 1e-9)), 2 * w))


def es_kernel(z, beta):
    """phi_beta(z), Sec. 3 Eq. (es), vectorised in numpy."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    inside = np.abs(z) <= 1.0
    zz = z[inside]
    out[inside] = np.exp(beta * (np.sqrt(1.0 - zz * zz) - 1.0))
    return out


def phihat(xi, beta: float, nquad: int = 200):
    """Fourier transform of the ES kernel, phihat(xi) = int_{-1}^{1} phi(z) cos(xi z) dz.

    Sec. 3.1 step 3 builds the correction factors from values of phihat but
    leaves open how those values are obtained.  phi has a
    square-root edge at |z| = 1, which slows Gauss-Legendre in z to algebraic
    convergence, so the integral is taken in theta with z = sin(theta):
      phihat(xi) = int_{-pi/2}^{pi/2} exp(beta (cos t - 1)) cos(xi sin t) cos t dt,
    an analytic integrand, by nquad-point Gauss-Legendre quadrature.
    """
    nodes, weights = np.polynomial.legendre.leggauss(nquad)
    t = 0.5 * math.pi * nodes
    wt = 0.5 * math.pi * weights * np.exp(beta * (np.cos(t) - 1.0)) * np.cos(t)
    xi = np.asarray(xi, dtype=np.float64)
    return np.cos(np.multiply.outer(xi, np.sin(t))) @ wt


def modes_1d(N: int):
    """Frequencies of I_N in output order: -floor(N/2) .. ceil(N/2)-1 (Eq. I)."""
    return np.arange(N, dtype=np.int64) - N // 2


def correction_1d(N: int, n: int, w: int, beta: float, nquad: int = 200):
    """Per-axis factor of p_k (Sec. 3.1 step 3): (2/w) / phihat(alpha k) * (-1)^k.

    alpha = w pi / n.  The (-1)^k factor comes from the grid origin: the fine
    grid point l sits at -pi + l h (the bin rule of Sec. 4.1), so the FFT of the
    spread grid carries e^{i k pi} relative to the paper's l h placement.
    """
    k = modes_1d(N)
    alpha = w * math.pi / n
    sgn = np.where(k % 2 == 0, 1.0, -1.0)
    return (2.0 / w) * sgn / phihat(alpha * k, beta, nquad)


class Params:
    """Plan parameters of Sec. 3 for one transform."""

    def __init__(self, N, eps, sigma=2.0, w=None):
        self.N = tuple(int(v) for v in N)
        self.dim = len(self.N)
        self.eps = float(eps)
        self.sigma = float(sigma)
        self.w = int(w) if w is not None else kernel_width(eps, sigma)
        self.beta = kernel_beta(self.w, sigma)
        self.n = tuple(fine_grid_size(v, self.w, sigma) for v in self.N)


# ---------------------------------------------------------------------------
# O1: exact sums
# ---------------------------------------------------------------------------
def _coords(pts):
    pts = [np.ascontiguousarray(np.asarray(p, dtype=np.float64)) for p in pts]
    M = pts[0].shape[0]
    for p in pts:
        if p.shape != (M,):
            raise ValueError("coordinate arrays must be 1-D of equal length")
    return pts, M


def _y(pts):
    """The second coordinate array, or None in 1D."""
    return pts[1] if len(pts) >= 2 else None


def direct_type1(pts, c, N, iflag=+1, modes=None):
    """f_k = sum_j c_j exp(i iflag k.x_j) (Eq. 2d1 with sign iflag).

    pts: list of d coordinate arrays; c: complex (M,); N: d mode counts.
    modes: optional flat mode indices (k1 fastest); default all, returned with
    shape (N3, N2, N1) / (N2, N1).
    """
    pts, M = _coords(pts)
    dim = len(pts)
    c = np.ascontiguousarray(np.asarray(c, dtype=np.complex128))
    Nv = np.asarray(N, dtype=np.int64)
    if modes is None:
        nk = int(np.prod(Nv))
        kl = None
    else:
        kl = np.ascontiguousarray(np.asarray(modes, dtype=np.int64))
        nk = kl.shape[0]
    f = np.zeros(nk, dtype=np.complex128)
    z = pts[2] if dim == 3 else None
    _load().orc_direct_type1(dim, M, _ptr(pts[0]), _ptr(_y(pts)), _ptr(z), _ptr(c),
                             int(iflag), _ptr(Nv), nk, _ptr(kl), _ptr(f))
    if modes is None:
        return f.reshape(tuple(reversed(tuple(int(v) for v in N))))
    return f


def direct_type2(pts, f, iflag=+1, targets=None):
    """c_j = sum_k f_k exp(-i iflag k.x_j) (Eq. 2d2; type 2 takes the sign opposite to type 1).

    f: complex array of shape (N2, N1) or (N3, N2, N1).  targets: optional
    point indices; default all M.
    """
    pts, M = _coords(pts)
    dim = len(pts)
    f = np.ascontiguousarray(np.asarray(f, dtype=np.complex128))
    N = tuple(reversed(f.shape))
    Nv = np.asarray(N, dtype=np.int64)
    if targets is None:
        nt = M
        jl = None
    else:
        jl = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
        nt = jl.shape[0]
    c = np.zeros(nt, dtype=np.complex128)
    z = pts[2] if dim == 3 else None
    _load().orc_direct_type2(dim, M, _ptr(pts[0]), _ptr(_y(pts)), _ptr(z), _ptr(f),
                             int(iflag), _ptr(Nv), nt, _ptr(jl), _ptr(c))
    return c


def direct_type3(pts, c, freqs, iflag=+1):
    """f_k = sum_j c_j exp(i iflag s_k.x_j) at real frequencies s_k: the type 3
    (nonuniform to nonuniform) transform the paper names as future work, by its
    definition.  pts and freqs: lists of d arrays (M and K entries)."""
    pts, M = _coords(pts)
    fr, K = _coords(freqs)
    dim = len(pts)
    if len(fr) != dim:
        raise ValueError("points and frequencies must have the same dimension")
    c = np.ascontiguousarray(np.asarray(c, dtype=np.complex128))
    f = np.zeros(K, dtype=np.complex128)
    z = pts[2] if dim == 3 else None
    u = fr[2] if dim == 3 else None
    _load().orc_direct_type3(dim, M, _ptr(pts[0]), _ptr(_y(pts)), _ptr(z), _ptr(c), int(iflag),
                             K, _ptr(fr[0]), _ptr(_y(fr)), _ptr(u), _ptr(f))
    return f


# ---------------------------------------------------------------------------
# O2: the three-step algorithm of Sec. 3 in FP64
# ---------------------------------------------------------------------------
def spread(pts, c, n, w, beta):
    """Sec. 3.1 step 1: fine grid b of shape (n2, n1) / (n3, n2, n1)."""
    pts, M = _coords(pts)
    dim = len(pts)
    c = np.ascontiguousarray(np.asarray(c, dtype=np.complex128))
    nv = np.asarray(n, dtype=np.int64)
    b = np.zeros(tuple(reversed(tuple(int(v) for v in n))), dtype=np.complex128)
    z = pts[2] if dim == 3 else None
    _load().orc_spread(dim, M, _ptr(pts[0]), _ptr(_y(pts)), _ptr(z), _ptr(c), _ptr(nv),
                       int(w), float(beta), _ptr(b))
    return b


def interp(pts, b, w, beta):
    """Sec. 3.2 step 3: values c_j interpolated from the fine grid b."""
    pts, M = _coords(pts)
    dim = len(pts)
    b = np.ascontiguousarray(np.asarray(b, dtype=np.complex128))
    n = tuple(reversed(b.shape))
    nv = np.asarray(n, dtype=np.int64)
    c = np.zeros(M, dtype=np.complex128)
    z = pts[2] if dim == 3 else None
    _load().orc_interp(dim, M, _ptr(pts[0]), _ptr(_y(pts)), _ptr(z), _ptr(b), _ptr(nv),
                       int(w), float(beta), _ptr(c))
    return c


def _fft_signed(a, sign):
    """Unnormalised d-D DFT with exponent sign `sign` (Sec. 3.1 step 2, 3.2 step 2)."""
    if sign > 0:
        return np.fft.ifftn(a, norm="forward")
    return np.fft.fftn(a, norm="backward")


def _mode_index(N, n):
    """Fine-grid indices (k mod n) of the modes, one array per axis, slow axis first."""
    return np.ix_(*[np.mod(modes_1d(Ni), ni) for Ni, ni in reversed(list(zip(N, n)))])


def _correction(P, nquad=200):
    """Separable correction p_k on the (N_d, .., N_1) mode array (Sec. 3.1 step 3)."""
    facs = [correction_1d(Ni, ni, P.w, P.beta, nquad) for Ni, ni in zip(P.N, P.n)]
    out = facs[0]
    if P.dim >= 2:
        out = out[None, :] * facs[1][:, None]
    if P.dim == 3:
        out = out[None, :, :] * facs[2][:, None, None]
    return out


def nufft_type1(pts, c, N, eps=None, iflag=+1, w=None, sigma=2.0):
    """Type 1 by spreading, FFT and correction (Sec. 3.1), all in FP64.

    Give either eps (w from Sec. 3) or an explicit width w.
    """
    P = Params(N, eps if eps is not None else 1e-14, sigma, w)
    b = spread(pts, c, P.n, P.w, P.beta)
    bh = _fft_signed(b, iflag)
    return bh[_mode_index(P.N, P.n)] * _correction(P)


def nufft_type2(pts, f, eps=None, iflag=+1, w=None, sigma=2.0):
    """Type 2 by correction, zero-padding, inverse FFT and interpolation (Sec. 3.2)."""
    f = np.asarray(f, dtype=np.complex128)
    N = tuple(reversed(f.shape))
    P = Params(N, eps if eps is not None else 1e-14, sigma, w)
    bh = np.zeros(tuple(reversed(P.n)), dtype=np.complex128)
    bh[_mode_index(P.N, P.n)] = f * _correction(P)
    b = _fft_signed(bh, -iflag)
    return interp(pts, b, P.w, P.beta)


# ---------------------------------------------------------------------------
# O3: bin-sort (Sec. 4.1)
# ---------------------------------------------------------------------------
def cells(x, n):
    """Fine-grid cell l and fraction of each point along one axis (fixed-point rule)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    M = x.shape[0]
    cell = np.zeros(M, dtype=np.int64)
    frac = np.zeros(M, dtype=np.float64)
    _load().orc_cells(M, _ptr(x), int(n), _ptr(cell), _ptr(frac))
    return cell, frac


def binsort(pts, n, m):
    """Stable bin-sort: returns (bin index per point, counts per bin, permutation t)."""
    pts, M = _coords(pts)
    dim = len(pts)
    nv = np.asarray(n, dtype=np.int64)
    mv = np.asarray(m, dtype=np.int64)
    nb = [(int(a) + int(b) - 1) // int(b) for a, b in zip(n, m)]
    nbins = int(np.prod(nb))
    binidx = np.zeros(M, dtype=np.int64)
    counts = np.zeros(max(nbins, 1), dtype=np.int64)
    t = np.zeros(M, dtype=np.int64)
    z = pts[2] if dim == 3 else None
    _load().orc_binsort(dim, M, _ptr(pts[0]), _ptr(_y(pts)), _ptr(z), _ptr(nv), _ptr(mv),
                        _ptr(binidx), _ptr(counts), _ptr(t))
    return binidx, counts[:nbins], t


def subproblems(counts, msub):
    """Sec. 4.1 SM step 1: each bin's points split into runs of at most msub.

    Returns an int64 array of rows (bin, start offset in t, count).
    """
    rows = []
    start = 0
    for b, cnt in enumerate(np.asarray(counts).tolist()):
        off = 0
        while off < cnt:
            take = min(msub, cnt - off)
            rows.append((b, start + off, take))
            off += take
        start += cnt
    return np.asarray(rows, dtype=np.int64).reshape(-1, 3)


def rel_l2(a, b):
    """Relative l2 error ||a - b|| / ||b|| over all entries (Sec. 5.3)."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
