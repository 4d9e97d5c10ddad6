"""The allocation-free bin-sort entry point against the plan-based one.

nufft_binsort_noalloc serves callers that cannot allocate device memory: it
keeps all of its scratch in one fixed array inside the library.  Its results
must equal what nufft_setpts computes (read back with nufft_get_sort), bit for
bit, on consecutive calls that reuse that array.  This file is collected last
so that a run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

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


def _plan_sort(nb, dim, N, eps, prec, pts):
    p = nb.Plan(1, N, eps, prec=prec, method="sm")
    p.setpts(*pts)
    t, bc, _ = p.sort()
    out = (p.params["nf"][:dim], p.params["bins"][:dim], t.clone(), bc.clone())
    torch.cuda.synchronize()
    p.close()
    return out


@pytest.mark.gpu
def test_noalloc_binsort_matches_setpts_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nb = _lib()
    cases = [
        # dim, N, M, eps, prec, kind
        (2, (100, 90), 300001, 1e-5, 0, "rand"),
        (3, (40, 36, 30), 150007, 1e-9, 1, "gauss"),
    ]
    for dim, N, M, eps, prec, kind in cases:     # two calls in a row share the scratch
        dt = np.float32 if prec == 0 else np.float64
        rd = torch.float32 if prec == 0 else torch.float64
        pts = [torch.from_numpy(a).to(rd).cuda()
               for a in wl.points(kind, dim, M, 4242 + dim, dt)]
        nf, bins, t_ref, bc_ref = _plan_sort(nb, dim, N, eps, prec, pts)
        nbins = bc_ref.numel()
        perm = torch.full((M,), -1, dtype=torch.int32, device="cuda")
        bincount = torch.full((nbins,), -1, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        nb.binsort_noalloc(dim, prec, M, nb._dptr(pts[0]), nb._dptr(pts[1]),
                           nb._dptr(pts[2]) if dim == 3 else None, nf, bins,
                           nb._dptr(perm), nb._dptr(bincount), stream.cuda_stream)
        torch.cuda.synchronize()
        assert torch.equal(perm, t_ref)
        assert torch.equal(bincount, bc_ref)
