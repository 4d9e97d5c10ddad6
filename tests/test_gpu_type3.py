"""GPU type 3 (nonuniform to nonuniform) against the exact sum of the FP64
oracle, f_k = sum_j c_j exp(i iflag s_k . x_j).

The paper gives no algorithm for type 3 (it lists type 3 as future work), so
the oracle is the definition itself.  The library computes it from two stages
of tolerance eps each (the type 1 spreading step and a type 2 transform), the
second one's error scaled by the correction 1/phihat at the band edge, which for
sigma = 2 and beta = 2.30 w is at most about e^{0.14 w} times its centre value
(<= 3 for w <= 8, <= 7 for w <= 14).  In single precision the rescaled
coordinates u = (x - C) / gamma and tau = t h are themselves rounded to single
precision: an RMS phase error of |t| times half an ulp of u, with |t| up to
S gamma ~ n / 4 per axis and ulp(u) <= 2^-22 (|u| < pi), i.e. about
2^-23 sqrt(sum_i (n_i / 4)^2) relative in the sum.  The bar is therefore
    relative l2 <= (2 + e^{0.14 w}) eps  [+ 2^-23 sqrt(sum_i (n_i / 4)^2) in single precision]
with n_i the spreading grid the plan reports.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_08463_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08463_gb300 import binding
    binding.load()
    return binding


def _bar(eps, w, prec, n=(1,)):
    base = (2.0 + math.exp(0.14 * w)) * eps
    if prec == 0:
        base += 2.0 ** -23 * math.sqrt(sum((v / 4.0) ** 2 for v in n))
    return base


def _uniform(seed, n, lo, hi, dt):
    return (lo + (hi - lo) * wl.uniform01(seed, n, stream=7)).astype(dt)


CASES = [
    # dim, M, K, x half-range, s half-range, eps, prec
    (1, 20001, 3001, 7.0, 60.0, 1e-6, 0),
    (1, 5003, 4001, 2.0, 800.0, 1e-10, 1),
    (2, 30011, 2003, 4.0, 25.0, 1e-5, 0),
    (2, 8009, 1501, 10.0, 8.0, 1e-9, 1),
    (3, 40009, 1201, 3.0, 10.0, 1e-4, 0),
    (3, 9001, 801, 2.5, 6.0, 1e-8, 1),
]


@pytest.mark.parametrize("dim,M,K,X,S,eps,prec", CASES)
@pytest.mark.parametrize("iflag", [+1, -1])
def test_type3_matches_exact_sum(nb, dim, M, K, X, S, eps, prec, iflag):
    dt = np.float32 if prec == 0 else np.float64
    ct = np.complex64 if prec == 0 else np.complex128
    # off-centre boxes: the library centres both sets itself
    xs = [_uniform(100 + d, M, -X + 0.7 * d, X + 0.7 * d, dt) for d in range(dim)]
    ss = [_uniform(200 + d, K, -S - 3.0 * d, S - 3.0 * d, dt) for d in range(dim)]
    c = wl.strengths(M, 300, ct)
    p = nb.Plan3(dim, eps, iflag=iflag, prec=prec)
    p.setpts([torch.from_numpy(a).cuda() for a in xs], [torch.from_numpy(a).cuda() for a in ss])
    f = p.execute(torch.from_numpy(c).cuda())
    torch.cuda.synchronize()
    got = f.cpu().numpy()
    ref = oracle.direct_type3([a.astype(np.float64) for a in xs], c.astype(np.complex128),
                              [a.astype(np.float64) for a in ss], iflag)
    e = oracle.rel_l2(got, ref)
    w, n = p.params["w"], p.params["nf"][:dim]
    bar = _bar(eps, w, prec, n)
    from conftest import record_exact_error
    record_exact_error("type3 %dD M=%d K=%d X=%g S=%g n=%s iflag=%+d" % (dim, M, K, X, S, n, iflag),
                       eps, e, float("nan"), bar)
    assert e <= bar, (e, eps, bar)
    p.close()


def test_type3_ntransf_and_reuse(nb):
    dim, M, K, nt, eps = 2, 6007, 907, 3, 1e-9
    xs = [_uniform(400 + d, M, -3.0, 3.0, np.float64) for d in range(dim)]
    c = wl.strengths(M, 401, np.complex128, ntransf=nt)
    p = nb.Plan3(dim, eps, ntransf=nt, prec=1)
    for rep, S in enumerate((5.0, 40.0)):          # new frequencies: the grid is resized
        ss = [_uniform(410 + rep * 3 + d, K, -S, S, np.float64) for d in range(dim)]
        p.setpts([torch.from_numpy(a).cuda() for a in xs], [torch.from_numpy(a).cuda() for a in ss])
        got = p.execute(torch.from_numpy(c).cuda()).cpu().numpy()
        for t in range(nt):
            ref = oracle.direct_type3(xs, c[t], ss, +1)
            assert oracle.rel_l2(got[t], ref) <= _bar(eps, p.params["w"], 1)
    p.close()


def test_type3_integer_frequencies_match_type1(nb):
    # at the integer frequencies of I_N and points in [-pi, pi), type 3 is type 1
    N, M, eps = (24, 20), 5001, 1e-9
    xs = wl.points("rand", 2, M, 500, np.float64)
    c = wl.strengths(M, 501, np.complex128)
    k = np.meshgrid(oracle.modes_1d(N[1]), oracle.modes_1d(N[0]), indexing="ij")
    ss = [k[1].ravel().astype(np.float64), k[0].ravel().astype(np.float64)]
    p3 = nb.Plan3(2, eps, prec=1)
    p3.setpts([torch.from_numpy(a).cuda() for a in xs], [torch.from_numpy(a).cuda() for a in ss])
    f3 = p3.execute(torch.from_numpy(c).cuda()).cpu().numpy()
    p1 = nb.Plan(1, N, eps, prec=1)
    p1.setpts(*[torch.from_numpy(a).cuda() for a in xs])
    f1 = p1.execute(c=torch.from_numpy(c).cuda()).cpu().numpy().ravel()
    exact = oracle.direct_type1(xs, c, N).ravel()
    assert oracle.rel_l2(f3, exact) <= _bar(eps, p3.params["w"], 1)
    assert oracle.rel_l2(f3, f1) <= 2 * _bar(eps, p3.params["w"], 1)
    p1.close()
    p3.close()


def test_type3_degenerate_sets(nb):
    eps = 1e-6
    p = nb.Plan3(1, eps, prec=0)
    # no points: f = 0
    p.setpts([torch.empty(0, device="cuda")], [torch.linspace(-3, 3, 11, device="cuda")])
    f = p.execute(torch.empty(0, dtype=torch.complex64, device="cuda"))
    torch.cuda.synchronize()
    assert torch.all(f == 0)
    # all points at one place, one frequency: a single exponential
    x = torch.full((5,), 0.3, device="cuda")
    s = torch.tensor([7.0], device="cuda")
    c = torch.ones(5, dtype=torch.complex64, device="cuda")
    p.setpts([x], [s])
    got = p.execute(c).cpu().numpy()
    assert abs(got[0] - 5 * np.exp(1j * 7.0 * 0.3)) < 5 * 2e-5
    # no frequencies: nothing to write
    p.setpts([x], [torch.empty(0, device="cuda")])
    p.execute(c, f=torch.empty(0, dtype=torch.complex64, device="cuda"))
    p.close()


def test_type3_errors(nb):
    from paper_2102_08463_gb300.binding import NufftError
    p = nb.Plan3(2, 1e-6, prec=0)
    x = torch.zeros(4, device="cuda")
    with pytest.raises(NufftError):      # a type 3 plan has no stage entry points
        nb.spread(p.handle, None)
    with pytest.raises(NufftError):      # non-finite coordinates
        p.setpts([x, torch.tensor([0.0, float("nan"), 0.0, 0.0], device="cuda")], [x, x])
    p.close()
    q = nb.Plan(1, (16, 16), 1e-6, prec=0)
    with pytest.raises(NufftError):      # nufft_setpts3 needs a type 3 plan
        nb.setpts3(q.handle, 0, None, None, None, 0, None, None, None)
    q.close()
