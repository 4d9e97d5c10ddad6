"""Batched execution (nufft_batch_*) against the same plans run one by one.

A heterogeneous batch -- 2D and 3D, type 1 and type 2, uneven N and M, single
and double precision, ntransf > 1, and a GM plan that the batch runs on its
own -- must reproduce each plan's own execute up to the reordering of atomic
additions (relative l2 <= 1e-5 single, 1e-12 double), both as a direct
batched execute and as a captured CUDA graph replayed twice.
"""
import numpy as np
import pytest

from paper_2102_08463_gb300 import workloads as wl

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SPECS = [
    # type, N, M, eps, prec, method, ntransf
    (1, (64, 48), 20000, 1e-5, 0, "sm", 1),
    (2, (64, 48), 15000, 1e-5, 0, "sm", 1),
    (1, (100, 90), 5000, 1e-5, 0, "sm", 2),
    (2, (33, 70), 7000, 1e-5, 0, "gmsort", 1),
    (1, (20, 18, 16), 30000, 1e-5, 0, "sm", 1),
    (2, (24, 16, 20), 12000, 1e-5, 0, "sm", 3),
    (1, (16, 16, 16), 9000, 1e-5, 0, "gmsort", 1),
    (1, (40, 40), 6000, 1e-9, 1, "sm", 1),
    (2, (12, 14, 10), 8000, 1e-9, 1, "sm", 1),
    (1, (48, 32), 4000, 1e-5, 0, "gm", 1),
    (1, (64, 48), 1, 1e-5, 0, "sm", 1),
]


def _rel(a, b):
    a = a.reshape(-1)
    b = b.reshape(-1)
    return float(torch.linalg.norm(a - b) / max(float(torch.linalg.norm(b)), 1e-300))


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08463_gb300 import binding
    binding.load()
    return binding


def test_batch_matches_individual_and_graph(nb):
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plans, cs, fs, refs = [], [], [], []
        for i, (tp, N, M, eps, prec, method, nt) in enumerate(SPECS):
            dim = len(N)
            dt = np.float32 if prec == 0 else np.float64
            ct = np.complex64 if prec == 0 else np.complex128
            rd = torch.float32 if prec == 0 else torch.float64
            p = nb.Plan(tp, N, eps, prec=prec, method=method, ntransf=nt, stream=stream)
            pts = [torch.from_numpy(a).to(rd).cuda() for a in wl.points("rand", dim, M, 500 + i, dt)]
            p.setpts(*pts)
            if tp == 1:
                c = torch.from_numpy(wl.strengths(M, 600 + i, ct, ntransf=nt)).cuda()
                ref = p.execute(c=c)
                f = torch.zeros_like(ref)
            else:
                f = torch.from_numpy(wl.modes(N, 700 + i, ct, ntransf=nt)).cuda()
                ref = p.execute(f=f)
                c = torch.zeros_like(ref)
            plans.append(p)
            cs.append(c)
            fs.append(f)
            refs.append(ref.clone())
        stream.synchronize()
        before = [r.clone() for r in refs]

        batch = nb.Batch(plans, stream=stream)
        for (tp, *_), c, f in zip(SPECS, cs, fs):
            (f if tp == 1 else c).zero_()
        batch.execute(cs, fs)
        stream.synchronize()
        for (tp, N, M, eps, prec, method, nt), c, f, ref in zip(SPECS, cs, fs, before):
            got = f if tp == 1 else c
            assert _rel(got, ref) < (1e-5 if prec == 0 else 1e-12), (tp, N, M, method)

        batch.capture(cs, fs)
        for _ in range(2):
            for (tp, *_), c, f in zip(SPECS, cs, fs):
                (f if tp == 1 else c).zero_()
            batch.launch()
            stream.synchronize()
            for (tp, N, M, eps, prec, method, nt), c, f, ref in zip(SPECS, cs, fs, before):
                got = f if tp == 1 else c
                assert _rel(got, ref) < (1e-5 if prec == 0 else 1e-12), (tp, N, M, method)
        batch.close()
        # the plans work on their own again after the batch is gone
        p0 = plans[0]
        again = p0.execute(c=cs[0])
        stream.synchronize()
        assert _rel(again, before[0]) < 1e-5
        for p in plans:
            p.close()


def test_batch_errors(nb):
    with pytest.raises(nb.NufftError):
        nb.Batch([])
