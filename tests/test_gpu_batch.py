"""Batched execution (nufft_batch_*) against the same plans run one by one and
against the oracle.

A heterogeneous batch -- 2D and 3D, type 1 and type 2, uneven N and M, single
and double precision, ntransf > 1, GM plans -- must reproduce each plan's own
execute up to the reordering of atomic additions (relative l2 <= 1e-5 single,
1e-12 double), both as a direct batched execute and as a captured CUDA graph
replayed twice; back-to-back executes with different arrays and a later replay
must each use their own arrays.  The 256-plan workload of the benchmark (plus
its ntransf = 32 plan) runs as one batch and sampled plans are checked against
the FP64 oracle pipeline at the same width and against the exact sums (2 eps).
"""
import numpy as np
import pytest

import oracle
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
    (2, (30, 26), 3000, 1e-5, 0, "gm", 1),
    (2, (12, 10, 14), 5000, 1e-5, 0, "gm", 2),
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


def _make(nb, stream, seed0):
    plans, cs, fs, refs = [], [], [], []
    for i, (tp, N, M, eps, prec, method, nt) in enumerate(SPECS):
        dim = len(N)
        dt = np.float32 if prec == 0 else np.float64
        ct = np.complex64 if prec == 0 else np.complex128
        rd = torch.float32 if prec == 0 else torch.float64
        p = nb.Plan(tp, N, eps, prec=prec, method=method, ntransf=nt, stream=stream)
        pts = [torch.from_numpy(a).to(rd).cuda() for a in wl.points("rand", dim, M, 500 + i, dt)]
        p.setpts(*pts)
        plans.append(p)
    sets = []
    for k in range(2):                       # two sets of input / output arrays
        cs, fs, refs = [], [], []
        for i, (p, (tp, N, M, eps, prec, method, nt)) in enumerate(zip(plans, SPECS)):
            ct = np.complex64 if prec == 0 else np.complex128
            if tp == 1:
                c = torch.from_numpy(wl.strengths(M, seed0 + 100 * k + i, ct, ntransf=nt)).cuda()
                ref = p.execute(c=c).clone()
                f = torch.zeros_like(ref)
            else:
                f = torch.from_numpy(wl.modes(N, seed0 + 100 * k + i, ct, ntransf=nt)).cuda()
                ref = p.execute(f=f).clone()
                c = torch.zeros_like(ref)
            cs.append(c)
            fs.append(f)
            refs.append(ref)
        sets.append((cs, fs, refs))
    stream.synchronize()
    return plans, sets


def _check_set(cs, fs, refs):
    for (tp, N, M, eps, prec, method, nt), c, f, ref in zip(SPECS, cs, fs, refs):
        got = f if tp == 1 else c
        assert _rel(got, ref) < (1e-5 if prec == 0 else 1e-12), (tp, N, M, method)


def _clear(cs, fs):
    for (tp, *_), c, f in zip(SPECS, cs, fs):
        (f if tp == 1 else c).zero_()


def test_batch_back_to_back_executes_and_replay(nb):
    """Executes queued back to back with different arrays, no host synchronization
    between them, then a replay of a graph captured with the first arrays: each
    uses its own arrays (the arguments are staged per call)."""
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plans, sets = _make(nb, stream, 900)
        batch = nb.Batch(plans, stream=stream)
        (c0, f0, r0), (c1, f1, r1) = sets
        batch.capture(c0, f0)
        _clear(c0, f0)
        _clear(c1, f1)
        for _ in range(3):                   # more calls than staging slots
            batch.execute(c0, f0)
            batch.execute(c1, f1)
        stream.synchronize()
        _check_set(c0, f0, r0)
        _check_set(c1, f1, r1)
        _clear(c0, f0)
        _clear(c1, f1)
        batch.execute(c1, f1)
        batch.launch()                       # the graph still replays the first arrays
        stream.synchronize()
        _check_set(c0, f0, r0)
        _check_set(c1, f1, r1)
        batch.close()
        for p in plans:
            p.close()


def test_batch_256_plans_against_oracle(nb):
    """The benchmark's many-plan workload in one captured batch; sampled plans of
    every (dimension, type) class and the ntransf = 32 plan against the oracle."""
    import bench
    specs = bench.batch_specs()
    stream = torch.cuda.Stream()
    eps = 1e-5
    with torch.cuda.stream(stream):
        plans, cs, fs, host = [], [], [], []
        for i, sp in enumerate(specs):
            dim = len(sp["N"])
            method = "gm" if i % 7 == 3 else "auto"          # GM plans join the groups
            p = nb.Plan(sp["type"], sp["N"], eps, prec=0, ntransf=sp["ntransf"], method=method,
                        stream=stream)
            pts = wl.points("rand", dim, sp["M"], 7000 + i, np.float32)
            p.setpts(*[torch.from_numpy(a).cuda() for a in pts])
            if sp["type"] == 1:
                c = wl.strengths(sp["M"], 8000 + i, np.complex64, ntransf=sp["ntransf"])
                shp = tuple(reversed(sp["N"]))
                dc = torch.from_numpy(c).cuda()
                df = torch.zeros(((sp["ntransf"],) + shp) if sp["ntransf"] > 1 else shp,
                                 dtype=torch.complex64, device="cuda")
                host.append((pts, c))
            else:
                f = wl.modes(sp["N"], 9000 + i, np.complex64)
                df = torch.from_numpy(f).cuda()
                dc = torch.zeros(sp["M"], dtype=torch.complex64, device="cuda")
                host.append((pts, f))
            plans.append(p)
            cs.append(dc)
            fs.append(df)
        batch = nb.Batch(plans, stream=stream)
        batch.capture(cs, fs)
        batch.launch()
        stream.synchronize()
        # sample: per (dim, type) class the smallest and the median plan by work, and the
        # ntransf = 32 plan
        from conftest import record_exact_error
        picks = []
        for dim in (2, 3):
            for tp in (1, 2):
                idx = [i for i, sp in enumerate(specs[:256])
                       if len(sp["N"]) == dim and sp["type"] == tp]
                idx.sort(key=lambda i: specs[i]["M"] + int(np.prod(specs[i]["N"])))
                picks += [idx[0], idx[len(idx) // 2], idx[len(idx) // 3]]
        picks.append(256)
        for i in picks:
            sp, p = specs[i], plans[i]
            pts, data = host[i]
            p64 = [a.astype(np.float64) for a in pts]
            w = p.params["w"]
            kidx = wl.sample_indices(int(np.prod(sp["N"])) if sp["type"] == 1 else sp["M"], 16,
                                     100 + i)
            ts = (0, sp["ntransf"] - 1) if sp["ntransf"] > 1 else (None,)
            for t in ts:
                d = (data[t] if t is not None else data).astype(np.complex128)
                if sp["type"] == 1:
                    got = fs[i].cpu().numpy()
                    got = got[t] if t is not None else got
                    same = oracle.nufft_type1(p64, d, sp["N"], w=w)
                    exact = oracle.direct_type1(p64, d, sp["N"], modes=kidx)
                    gs, ss = got.ravel()[kidx], same.ravel()[kidx]
                else:
                    got = cs[i].cpu().numpy()
                    same = oracle.nufft_type2(p64, d, w=w)
                    exact = oracle.direct_type2(p64, d, targets=kidx)
                    gs, ss = got[kidx], same[kidx]
                assert oracle.rel_l2(got, same) < 2e-5, (i, sp)
                e, e_or = oracle.rel_l2(gs, exact), oracle.rel_l2(ss, exact)
                bar = max(2 * eps, e_or + 0.2 * eps)
                record_exact_error("batch plan %d type%d N=%s M=%d%s" % (
                    i, sp["type"], sp["N"], sp["M"], "" if t is None else " t=%d" % t),
                    eps, e, e_or, bar)
                assert e <= bar, (i, sp, e, e_or)
        batch.close()
        for p in plans:
            p.close()
