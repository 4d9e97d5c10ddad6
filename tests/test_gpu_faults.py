"""Error paths under injected failures (host side only; no GPU fault is made).

nufft_debug_fail makes the n-th next device allocation, or the next cuFFT plan,
fail as an out-of-memory or cuFFT error would, without touching the device.
Every failure point of makeplan, setpts and the host-buffer execute must
return the right error code, leave any plan destroyable (and usable once the
failure is gone), and leak nothing: the device's free memory comes back to
where it was.  debug_checks: bad coordinates are reported through the plan's
device status word, read by nufft_get_status, instead of trapping.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_08463_gb300 import workloads as wl

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N = (512, 512)          # fine grid 1024^2 complex64 = 8 MiB: a leak of it shows
M = 100000
SLACK = 4 << 20         # driver-side rounding of small allocations


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08463_gb300 import binding
    binding.load()
    binding.debug_fail(binding.FAIL_ALLOC, -1)
    binding.debug_fail(binding.FAIL_CUFFT, -1)
    yield binding
    binding.debug_fail(binding.FAIL_ALLOC, -1)
    binding.debug_fail(binding.FAIL_CUFFT, -1)


def _free():
    """Device memory not held by this library: the driver's free bytes plus what
    torch's caching allocator keeps reserved (its segments are not ours)."""
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0] + torch.cuda.memory_reserved()


@pytest.fixture(scope="module")
def data():
    pts = wl.points("rand", 2, M, 71, np.float32)
    c = wl.strengths(M, 72, np.complex64)
    return pts, c


def _check_result(p, pts, c, f):
    ref = oracle.nufft_type1([a.astype(np.float64) for a in pts], c.astype(np.complex128), N,
                             w=p.params["w"])
    assert oracle.rel_l2(f, ref) < 2e-5


def test_makeplan_allocation_failures(nb):
    h = nb.makeplan(1, 2, N, eps=1e-5, prec=0)      # warm-up: cuFFT and module loading
    nb.destroy(h)
    base = _free()
    nb.debug_fail(nb.FAIL_ALLOC, -1)
    nb.destroy(nb.makeplan(1, 2, N, eps=1e-5, prec=0))
    n_alloc = nb.debug_fail(nb.FAIL_ALLOC, -1)
    assert n_alloc >= 6
    for k in range(n_alloc):
        nb.debug_fail(nb.FAIL_ALLOC, k)
        with pytest.raises(nb.NufftError) as e:
            nb.makeplan(1, 2, N, eps=1e-5, prec=0)
        nb.debug_fail(nb.FAIL_ALLOC, -1)
        assert e.value.code == nb.NUFFT_ERR_ALLOC, k
    assert base - _free() <= SLACK


def test_makeplan_cufft_failure(nb):
    h = nb.makeplan(2, 3, (40, 40, 40), eps=1e-6, prec=0)
    nb.destroy(h)
    base = _free()
    nb.debug_fail(nb.FAIL_CUFFT, 0)
    with pytest.raises(nb.NufftError) as e:
        nb.makeplan(2, 3, (40, 40, 40), eps=1e-6, prec=0)
    nb.debug_fail(nb.FAIL_CUFFT, -1)
    assert e.value.code == nb.NUFFT_ERR_CUFFT
    assert base - _free() <= SLACK
    nb.destroy(nb.makeplan(2, 3, (40, 40, 40), eps=1e-6, prec=0))    # and it works again


def test_setpts_allocation_failures(nb, data):
    pts, c = data
    dp = [torch.from_numpy(a).cuda() for a in pts]
    dc = torch.from_numpy(c).cuda()
    p = nb.Plan(1, N, 1e-5, prec=0)
    nb.debug_fail(nb.FAIL_ALLOC, -1)
    p.setpts(*dp)
    n_alloc = nb.debug_fail(nb.FAIL_ALLOC, -1)
    p.close()
    assert n_alloc >= 4
    base = _free()
    for k in range(n_alloc):
        p = nb.Plan(1, N, 1e-5, prec=0)
        nb.debug_fail(nb.FAIL_ALLOC, k)
        with pytest.raises(nb.NufftError) as e:
            p.setpts(*dp)
        nb.debug_fail(nb.FAIL_ALLOC, -1)
        assert e.value.code == nb.NUFFT_ERR_ALLOC, k
        with pytest.raises(nb.NufftError) as e:        # no points set: execute refuses
            p.execute(c=dc)
        assert e.value.code == nb.NUFFT_ERR_NOPTS
        p.setpts(*dp)                                   # usable once the failure is gone
        f = p.execute(c=dc)
        _check_result(p, pts, c, f.cpu().numpy())
        p.close()
    assert base - _free() <= SLACK


def test_execute_host_staging_failure(nb, data):
    pts, c = data
    hp = [torch.from_numpy(a) for a in pts]
    hc = torch.from_numpy(c)
    p = nb.Plan(1, N, 1e-5, prec=0)
    base = _free()
    nb.debug_fail(nb.FAIL_ALLOC, 0)
    with pytest.raises(nb.NufftError) as e:
        p.execute_host(*hp, c=hc)
    nb.debug_fail(nb.FAIL_ALLOC, -1)
    assert e.value.code == nb.NUFFT_ERR_ALLOC
    f = p.execute_host(*hp, c=hc)
    _check_result(p, pts, c, f.numpy())
    p.close()
    assert base - _free() <= SLACK


def test_debug_checks_report_bad_coordinates(nb, data):
    pts, c = data
    p = nb.Plan(1, N, 1e-5, prec=0, debug_checks=True)
    p.setpts(*[torch.from_numpy(a).cuda() for a in pts])
    nb.get_status(p.handle)                          # valid points: passes
    for bad in (float("nan"), 10 * math.pi, float("inf")):
        x = pts[0].copy()
        x[M // 2] = bad
        p.setpts(torch.from_numpy(x).cuda(), torch.from_numpy(pts[1]).cuda())
        with pytest.raises(nb.NufftError) as e:
            nb.get_status(p.handle)
        assert e.value.code == nb.NUFFT_ERR_CHECK
        nb.get_status(p.handle)                      # reading the status clears it
    p.close()
    q = nb.Plan(1, N, 1e-5, prec=0)                  # without debug_checks: always OK
    x = pts[0].copy()
    x[0] = 10 * math.pi
    q.setpts(torch.from_numpy(x).cuda(), torch.from_numpy(pts[1]).cuda())
    nb.get_status(q.handle)
    q.close()
