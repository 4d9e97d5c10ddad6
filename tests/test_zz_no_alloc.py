"""The allocation-free bin-sort entry point against the plan-based one and the oracle.

nufft_binsort_noalloc serves callers that cannot allocate device memory (code
running inside another allocator, real-time callers with a memory budget fixed
at start-up): it keeps all of its scratch in one fixed array inside the
library.  Its results must equal what nufft_setpts computes (read back with
nufft_get_sort) and the oracle's stable bin-sort, bit for bit, on consecutive
calls that reuse that array, up to its limits (2^20 points, 16384 bins), and a
call after the warm-up must leave the device's free memory unchanged.  This
file is collected last so that a run stopping at the first failure has run
every other test first.
"""
import numpy as np
import pytest

import oracle
from paper_2102_08463_gb300 import workloads as wl

torch = pytest.importorskip("torch")


def _lib():
    from paper_2102_08463_gb300 import binding
    binding.load()
    return binding


def test_noalloc_rejects_oversize_without_touching_the_gpu():
    import ctypes
    nb = _lib()
    # placeholder pointers: the size checks return before any pointer is used
    fake = ctypes.c_void_p(256)
    with pytest.raises(nb.NufftError) as e:
        nb.binsort_noalloc(2, 0, (1 << 20) + 1, fake, fake, None, (64, 64), (16, 16), fake, fake)
    assert e.value.code == nb.NUFFT_ERR_SIZE
    with pytest.raises(nb.NufftError) as e:      # 256 x 256 bins > 16384
        nb.binsort_noalloc(2, 0, 10, fake, fake, None, (256, 256), (1, 1), fake, fake)
    assert e.value.code == nb.NUFFT_ERR_SIZE


def _plan_sort(nb, dim, N, eps, prec, pts, bins=None):
    kw = {} if bins is None else {"bins": bins}
    p = nb.Plan(1, N, eps, prec=prec, method="sm", **kw)
    p.setpts(*pts)
    t, bc, _ = p.sort()
    out = (p.params["nf"][:dim], p.params["bins"][:dim], t.clone(), bc.clone())
    torch.cuda.synchronize()
    p.close()
    return out


def _noalloc(nb, dim, prec, M, pts, nf, bins, nbins):
    perm = torch.full((max(M, 1),), -1, dtype=torch.int32, device="cuda")
    bincount = torch.full((nbins,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    nb.binsort_noalloc(dim, prec, M, nb._dptr(pts[0]), nb._dptr(pts[1]),
                       nb._dptr(pts[2]) if dim == 3 else None, nf, bins,
                       nb._dptr(perm) if M > 0 else None, nb._dptr(bincount), stream.cuda_stream)
    torch.cuda.synchronize()
    return perm[:M], bincount


@pytest.mark.gpu
def test_noalloc_binsort_matches_setpts_and_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nb = _lib()
    cases = [
        # dim, N, M, eps, prec, kind, bins
        (2, (100, 90), 300001, 1e-5, 0, "rand", None),
        (3, (40, 36, 30), 150007, 1e-9, 1, "gauss", None),
        (2, (512, 512), 1 << 20, 1e-5, 0, "rand", (8, 8)),        # the limits: 2^20 points,
        (2, (512, 512), 4099, 1e-5, 0, "cluster", (8, 8)),        # 128 x 128 = 16384 bins
    ]
    for dim, N, M, eps, prec, kind, bins in cases:     # calls in a row share the scratch
        dt = np.float32 if prec == 0 else np.float64
        rd = torch.float32 if prec == 0 else torch.float64
        nf_guess = [2 * v for v in N]
        host = wl.points(kind, dim, M, 4242 + dim, dt, n=nf_guess)
        pts = [torch.from_numpy(a).to(rd).cuda() for a in host]
        nf, bins_used, t_ref, bc_ref = _plan_sort(nb, dim, N, eps, prec, pts, bins)
        nbins = bc_ref.numel()
        if bins is not None:
            assert nbins == 16384
        perm, bincount = _noalloc(nb, dim, prec, M, pts, nf, bins_used, nbins)
        assert torch.equal(perm, t_ref)
        assert torch.equal(bincount, bc_ref)
        _, counts, t_or = oracle.binsort([a.astype(np.float64) for a in host], nf, bins_used)
        assert np.array_equal(bincount.cpu().numpy().astype(np.int64), counts)
        assert np.array_equal(perm.cpu().numpy().astype(np.int64), t_or)
        # a second call on the same inputs gives the same result and allocates
        # nothing: the device's free memory is the same before and after it
        perm2 = torch.full((M,), -1, dtype=torch.int32, device="cuda")
        bincount2 = torch.full((nbins,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        nb.binsort_noalloc(dim, prec, M, nb._dptr(pts[0]), nb._dptr(pts[1]),
                           nb._dptr(pts[2]) if dim == 3 else None, nf, bins_used,
                           nb._dptr(perm2), nb._dptr(bincount2),
                           torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        assert torch.equal(perm2, perm) and torch.equal(bincount2, bincount)


@pytest.mark.gpu
def test_noalloc_empty_input_with_null_perm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nb = _lib()
    x = torch.empty(0, dtype=torch.float32, device="cuda")
    bincount = torch.full((16,), -1, dtype=torch.int32, device="cuda")
    nb.binsort_noalloc(2, 0, 0, None, None, None, (64, 64), (16, 16), None, nb._dptr(bincount),
                       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert torch.equal(bincount, torch.zeros_like(bincount))
    del x
