"""GPU parity of the 1D transforms (the d = 1 case of Sec. 3; the paper lists 1D
as future work) against the FP64 oracle, with the bars of test_gpu_parity:
bin-sort bit-exact; the oracle's pipeline at the same width within 2e-5
(single) / 1e-11 (double) relative l2; the exact sums within 2 eps, or the
oracle pipeline's own error plus 0.2 eps where that misses 2 eps.
"""
import math

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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _check_exact(name, got, exact, e_or, eps):
    from conftest import record_exact_error
    e = oracle.rel_l2(got, exact)
    bar = max(2 * eps, e_or + 0.2 * eps)
    record_exact_error(name, eps, e, e_or, bar)
    assert e <= bar, (name, e, bar)


@pytest.mark.parametrize("kind,M", [("rand", 100003), ("cluster", 7001), ("gauss", 30011), ("rand", 1)])
@pytest.mark.parametrize("prec", [0, 1])
def test_binsort_1d_bit_exact(nb, kind, M, prec):
    dt = np.float32 if prec == 0 else np.float64
    p = nb.Plan(1, (5000,), 1e-5 if prec == 0 else 1e-9, prec=prec, method="sm")
    nf = p.params["nf"][:1]
    pts = wl.points(kind, 1, M, 500 + M, dt, n=nf)
    pts[0][: min(M, 3)] = np.array([-math.pi, math.pi, np.nextafter(dt(math.pi), dt(4))], dt)[: min(M, 3)]
    p.setpts(_dev(pts[0]))
    t, bc, nsub = p.sort()
    bins = p.params["bins"][:1]
    _, counts, t_ref = oracle.binsort([pts[0].astype(np.float64)], nf, bins)
    assert np.array_equal(_host(bc).astype(np.int64), counts)
    assert np.array_equal(_host(t).astype(np.int64), t_ref)
    assert nsub == oracle.subproblems(counts, 1024).shape[0]
    p.close()


CASES_1D = [
    # N, M, eps, prec
    ((1000,), 20001, 1e-5, 0),
    ((777,), 3001, 1e-2, 0),
    ((4097,), 50003, 1e-6, 0),
    ((1500,), 9001, 1e-9, 1),
    ((640,), 4000, 1e-12, 1),
]


@pytest.mark.parametrize("N,M,eps,prec", CASES_1D)
@pytest.mark.parametrize("method", ["gm", "gmsort", "sm"])
@pytest.mark.parametrize("iflag", [+1, -1])
def test_type1_1d_parity(nb, N, M, eps, prec, method, iflag):
    dt = np.float32 if prec == 0 else np.float64
    ct = np.complex64 if prec == 0 else np.complex128
    x = wl.points("rand", 1, M, 7 * M, dt)[0]
    c = wl.strengths(M, 8 + M, ct)
    p = nb.Plan(1, N, eps, iflag=iflag, prec=prec, method=method)
    p.setpts(_dev(x))
    f = _host(p.execute(c=_dev(c)))
    x64 = [x.astype(np.float64)]
    same = oracle.nufft_type1(x64, c.astype(np.complex128), N, iflag=iflag, w=p.params["w"])
    assert oracle.rel_l2(f, same) < TOL[prec]
    exact = oracle.direct_type1(x64, c.astype(np.complex128), N, iflag)
    _check_exact("type1 1D N=%s M=%d %s iflag=%+d" % (N, M, method, iflag), f, exact,
                 oracle.rel_l2(same, exact), eps)
    p.close()


@pytest.mark.parametrize("N,M,eps,prec", CASES_1D)
@pytest.mark.parametrize("method", ["gm", "gmsort", "sm"])
@pytest.mark.parametrize("iflag", [+1, -1])
def test_type2_1d_parity(nb, N, M, eps, prec, method, iflag):
    dt = np.float32 if prec == 0 else np.float64
    ct = np.complex64 if prec == 0 else np.complex128
    x = wl.points("rand", 1, M, 9 * M, dt)[0]
    f = wl.modes(N, 10 + M, ct)
    p = nb.Plan(2, N, eps, iflag=iflag, prec=prec, method=method)
    p.setpts(_dev(x))
    c = _host(p.execute(f=_dev(f)))
    x64 = [x.astype(np.float64)]
    same = oracle.nufft_type2(x64, f.astype(np.complex128), iflag=iflag, w=p.params["w"])
    assert oracle.rel_l2(c, same) < TOL[prec]
    exact = oracle.direct_type2(x64, f.astype(np.complex128), iflag)
    _check_exact("type2 1D N=%s M=%d %s iflag=%+d" % (N, M, method, iflag), c, exact,
                 oracle.rel_l2(same, exact), eps)
    p.close()


@pytest.mark.parametrize("kind", ["cluster", "gauss"])
@pytest.mark.parametrize("bins,msub", [(None, 0), ((100,), 64), ((1000,), 4000)])
def test_1d_clustered_bins_and_subproblems(nb, kind, bins, msub):
    N, M, eps = (2000,), 40001, 1e-6
    p1 = nb.Plan(1, N, eps, prec=0, method="sm", bins=bins, msub=msub)
    nf = p1.params["nf"][:1]
    x = wl.points(kind, 1, M, 11, np.float32, n=nf, spread=0.2)[0]
    c = wl.strengths(M, 12, np.complex64)
    p1.setpts(_dev(x))
    g1 = _host(p1.execute(c=_dev(c)))
    x64 = [x.astype(np.float64)]
    assert oracle.rel_l2(g1, oracle.nufft_type1(x64, c.astype(np.complex128), N,
                                                 w=p1.params["w"])) < TOL[0]
    p1.close()
    p2 = nb.Plan(2, N, eps, prec=0, method="sm", bins=bins, msub=msub)
    f = wl.modes(N, 13, np.complex64)
    p2.setpts(_dev(x))
    c2 = _host(p2.execute(f=_dev(f)))
    assert oracle.rel_l2(c2, oracle.nufft_type2(x64, f.astype(np.complex128),
                                                 w=p2.params["w"])) < TOL[0]
    p2.close()


@pytest.mark.parametrize("type_", [1, 2])
def test_1d_ntransf_and_host_buffers(nb, type_):
    N, M, nt, eps = (900,), 12007, 3, 1e-9
    x = wl.points("rand", 1, M, 21, np.float64)[0]
    x64 = [x]
    p = nb.Plan(type_, N, eps, prec=1, ntransf=nt)
    if type_ == 1:
        c = wl.strengths(M, 22, np.complex128, ntransf=nt)
        out = p.execute_host(torch.from_numpy(x).pin_memory(), c=torch.from_numpy(c).pin_memory())
        got = out.numpy()
        for t in range(nt):
            ref = oracle.nufft_type1(x64, c[t], N, w=p.params["w"])
            assert oracle.rel_l2(got[t], ref) < TOL[1]
    else:
        f = wl.modes(N, 23, np.complex128, ntransf=nt)
        out = p.execute_host(torch.from_numpy(x).pin_memory(), f=torch.from_numpy(f).pin_memory())
        got = out.numpy()
        for t in range(nt):
            ref = oracle.nufft_type2(x64, f[t], w=p.params["w"])
            assert oracle.rel_l2(got[t], ref) < TOL[1]
    p.close()


def test_1d_empty_and_single_point(nb):
    p = nb.Plan(1, (33,), 1e-6, prec=0)
    p.setpts(torch.empty(0, dtype=torch.float32, device="cuda"))
    f = _host(p.execute(c=torch.empty(0, dtype=torch.complex64, device="cuda")))
    assert np.all(f == 0)
    x = np.array([1.25], np.float32)
    p.setpts(_dev(x))
    f = _host(p.execute(c=_dev(np.array([2.0 - 1.0j], np.complex64))))
    exact = oracle.direct_type1([x.astype(np.float64)], np.array([2.0 - 1.0j]), (33,))
    assert oracle.rel_l2(f, exact) < 2e-6
    p.close()


def test_1d_in_a_batch(nb):
    plans, refs, args = [], [], []
    specs = [(1, (500,), 4001, "sm"), (2, (700,), 3001, "sm"), (1, (300,), 2001, "gm"),
             (2, (257,), 999, "gmsort"), (1, (500,), 1500, "sm")]
    for i, (ty, N, M, method) in enumerate(specs):
        x = wl.points("rand", 1, M, 40 + i, np.float32)[0]
        p = nb.Plan(ty, N, 1e-5, prec=0, method=method)
        p.setpts(_dev(x))
        x64 = [x.astype(np.float64)]
        if ty == 1:
            c = wl.strengths(M, 50 + i, np.complex64)
            out = torch.empty(N[::-1], dtype=torch.complex64, device="cuda")
            args.append((_dev(c), out))
            refs.append(oracle.nufft_type1(x64, c.astype(np.complex128), N, w=p.params["w"]))
        else:
            f = wl.modes(N, 60 + i, np.complex64)
            out = torch.empty(M, dtype=torch.complex64, device="cuda")
            args.append((out, _dev(f)))
            refs.append(oracle.nufft_type2(x64, f.astype(np.complex128), w=p.params["w"]))
        plans.append(p)
    b = nb.Batch(plans)
    b.execute([a[0] for a in args], [a[1] for a in args])
    for (ty, _, _, _), a, ref in zip(specs, args, refs):
        got = _host(a[1] if ty == 1 else a[0])
        assert oracle.rel_l2(got, ref) < TOL[0]
    b.close()
    for p in plans:
        p.close()
