"""The host-buffer execute (nufft_execute_host, the "total+mem" path of Sec. 5)
against the oracle.

Points, strengths and modes live in host memory (pinned or pageable); the call
copies them in, sorts, executes and copies the result out.  The host result must
match the oracle's FP64 pipeline at the same kernel width to rounding and the
exact sums within 2 eps (or the pipeline's own error + 0.2 eps where it misses
2 eps), on consecutive calls of different sizes that reuse and grow the plan's
staging.
"""
import numpy as np
import pytest

import oracle
from paper_2102_08463_gb300 import workloads as wl

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {0: 2e-5, 1: 1e-11}


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08463_gb300 import binding
    binding.load()
    return binding


def _host(a, pin):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.pin_memory() if pin else t


@pytest.mark.parametrize("pin", [True, False])
@pytest.mark.parametrize("type_", [1, 2])
@pytest.mark.parametrize("dim,N,eps,prec", [(2, (64, 48), 1e-5, 0), (3, (20, 16, 18), 1e-6, 0),
                                            (2, (40, 36), 1e-9, 1)])
def test_execute_host_matches_oracle(nb, pin, type_, dim, N, eps, prec):
    dt = np.float32 if prec == 0 else np.float64
    ct = np.complex64 if prec == 0 else np.complex128
    p = nb.Plan(type_, N, eps, prec=prec, stream=torch.cuda.Stream())
    w = p.params["w"]
    from conftest import record_exact_error
    for M in (3001, 9000, 500):             # the staging grows, then is reused
        seed = 31 * M + dim + type_
        pts = wl.points("rand", dim, M, seed, dt)
        hp = [_host(a, pin) for a in pts]
        p64 = [a.astype(np.float64) for a in pts]
        if type_ == 1:
            c = wl.strengths(M, seed + 1, ct)
            got = p.execute_host(*hp, c=_host(c, pin)).numpy()
            same = oracle.nufft_type1(p64, c.astype(np.complex128), N, w=w)
            exact = oracle.direct_type1(p64, c.astype(np.complex128), N)
        else:
            f = wl.modes(N, seed + 2, ct)
            got = p.execute_host(*hp, f=_host(f, pin)).numpy()
            same = oracle.nufft_type2(p64, f.astype(np.complex128), w=w)
            exact = oracle.direct_type2(p64, f.astype(np.complex128))
        assert oracle.rel_l2(got, same) < TOL[prec]
        e, e_or = oracle.rel_l2(got, exact), oracle.rel_l2(same, exact)
        bar = max(2 * eps, e_or + 0.2 * eps)
        record_exact_error("host type%d %dD N=%s M=%d %s" % (type_, dim, N, M,
                                                            "pinned" if pin else "pageable"),
                           eps, e, e_or, bar)
        assert e <= bar
    p.close()


def test_execute_host_ntransf(nb):
    N, M, nt = (32, 40), 2000, 3
    pts = wl.points("rand", 2, M, 5, np.float32)
    c = wl.strengths(M, 6, np.complex64, ntransf=nt)
    p = nb.Plan(1, N, 1e-5, prec=0, ntransf=nt)
    got = p.execute_host(*[_host(a, True) for a in pts], c=_host(c, True)).numpy()
    p64 = [a.astype(np.float64) for a in pts]
    for t in range(nt):
        ref = oracle.nufft_type1(p64, c[t].astype(np.complex128), N, w=p.params["w"])
        assert oracle.rel_l2(got[t], ref) < TOL[0]
    p.close()


def test_execute_host_empty(nb):
    p = nb.Plan(1, (16, 16), 1e-5, prec=0)
    e = torch.empty(0, dtype=torch.float32)
    f = p.execute_host(e, e, c=torch.empty(0, dtype=torch.complex64)).numpy()
    assert np.all(f == 0)
    p.close()
