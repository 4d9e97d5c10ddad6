"""Autotuner: the tuning cache on the CPU, and tuned tiles on the GPU."""
import numpy as np
import pytest

import oracle
from paper_2102_08463_gb300 import workloads as wl

torch = pytest.importorskip("torch")


def _lib():
    from paper_2102_08463_gb300 import binding
    binding.load()
    return binding


def test_tune_cache_file_roundtrip(tmp_path):
    nb = _lib()
    nb.tune_cache_clear()
    good = tmp_path / "cache.txt"
    good.write_text("# header\n1 2 0 6 200 22 0 3 16 16 1 1024 256 0.450000\n")
    nb.tune_cache_load(good)
    out = tmp_path / "out.txt"
    nb.tune_cache_save(out)
    lines = [l for l in out.read_text().splitlines() if not l.startswith("#")]
    assert lines == ["1 2 0 6 200 22 0 3 16 16 1 1024 256 0.450000"]
    bad = tmp_path / "bad.txt"
    bad.write_text("1 2 3\n")
    with pytest.raises(nb.NufftError):
        nb.tune_cache_load(bad)
    nb.tune_cache_clear()


@pytest.mark.gpu
def test_autotune_picks_the_fastest_and_plans_adopt_it(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nb = _lib()
    nb.tune_cache_clear()
    N, M, eps = (128, 128), 60000, 1e-5
    pts = wl.points("rand", 2, M, 31, np.float32)
    xd = [torch.from_numpy(a).cuda() for a in pts]
    c = torch.from_numpy(wl.strengths(M, 32, np.complex64)).cuda()
    f = torch.zeros((128, 128), dtype=torch.complex64, device="cuda")
    best, ms, trials = nb.autotune(1, N, eps, M, xd[0], xd[1], None, c, f, reps=2)
    assert len(trials) > 20
    assert ms == pytest.approx(min(t["exec_ms"] for t in trials))
    # a plan left on automatic tiles adopts the tuned ones for this problem class
    p = nb.Plan(1, N, eps)
    p.setpts(*xd)
    got = p.execute(c=c)
    prm = nb.get_params(p.handle)
    assert prm["method"] == best.method
    assert prm["bins"][:2] == tuple(best.bin)[:2]
    ref = oracle.nufft_type1([a.astype(np.float64) for a in pts],
                             c.cpu().numpy().astype(np.complex128), N, w=prm["w"])
    torch.cuda.synchronize()
    assert oracle.rel_l2(got.cpu().numpy(), ref) < 2e-5
    p.close()
    # the cache survives a save / clear / load cycle
    path = tmp_path / "tune.txt"
    nb.tune_cache_save(path)
    nb.tune_cache_clear()
    nb.tune_cache_load(path)
    q = nb.Plan(1, N, eps)
    q.setpts(*xd)
    assert nb.get_params(q.handle)["bins"][:2] == tuple(best.bin)[:2]
    q.close()
    nb.tune_cache_clear()
