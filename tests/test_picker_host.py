"""Host side of the learned tile picker (no GPU): the problem sampler keeps
its stated ranges, work bound and 80/20 split by seed, and a trial row turns
into one 12-feature row and a log2(ms) target per candidate, a trial timed at
sigma = 1.25 through that factor's kernel width and grid size."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def pk():
    from paper_2102_08463_gb300 import build, binding, picker
    build.build()
    binding.load()
    return picker


def test_sampler_is_deterministic_and_splits_by_seed(pk):
    a = pk.sample_problems(12, first_seed=0)
    b = pk.sample_problems(12, first_seed=0)
    assert a == b
    held = pk.sample_problems(6, first_seed=0, heldout=True)
    train = pk.sample_problems(6, first_seed=0, heldout=False)
    assert all(p["seed"] % 5 == 0 for p in held)
    assert all(p["seed"] % 5 != 0 for p in train)
    # the unfiltered draw is the union of the two splits, in seed order
    seeds = [p["seed"] for p in pk.sample_problems(40, first_seed=0)]
    assert seeds == sorted(seeds)


def test_sampled_problems_respect_ranges_and_work_bound(pk):
    for p in pk.sample_problems(60, first_seed=100):
        d = p["dim"]
        assert d in (2, 3) and p["type"] in (1, 2) and len(p["N"]) == d
        assert all(32 <= n <= 1024 for n in p["N"])
        assert 1e4 <= p["M"] <= 3e7 + 1
        assert 1e-12 <= p["eps"] <= 1e-2 * (1 + 1e-12)
        assert p["kind"] in ("rand", "gauss", "mixture")
        assert 0.01 * math.pi * (1 - 1e-12) <= p["spread"] <= 0.5 * math.pi * (1 + 1e-12)
        # single precision exactly where the tolerance allows it
        assert p["prec"] == (0 if p["eps"] >= 1e-6 else 1)
        # width rule of Sec. 3 at sigma = 2
        want_w = min(16, max(2, math.ceil(math.log10(1.0 / p["eps"]) - 1e-10) + 1))
        assert p["w"] == want_w
        assert p["M"] * p["w"] ** d * (16 if p["prec"] else 1) <= pk.MAX_WORK


def test_trial_row_features(pk):
    row = dict(seed=3, type=1, dim=2, N=[200, 120], M=50000, kind="rand", spread=0.3, eps=1e-5,
               prec=0, w=6, skew=0.25,
               trials=[[3, 10, 16, 1, 1024, 256, 0.5], [2, 16, 16, 1, 256, 128, 0.25],
                       [1, 16, 16, 1, 1024, 256, 2.0]])
    X, T = pk.features(row)
    assert X.shape == (3, 12) and X.dtype == np.float32
    assert np.allclose(T, [-1.0, -2.0, 1.0])
    # method one-hots: SM, GM-sort (neither), GM
    assert (X[0, 7], X[0, 8]) == (1.0, 0.0)
    assert (X[1, 7], X[1, 8]) == (0.0, 0.0)
    assert (X[2, 7], X[2, 8]) == (0.0, 1.0)
    # bin cells, M_sub and threads enter as log2 / 12, log2 / 12 and / 256
    assert X[0, 9] == pytest.approx(math.log2(160) / 12)
    assert X[1, 10] == pytest.approx(math.log2(256) / 12)
    assert X[1, 11] == pytest.approx(128 / 256)
    # problem features are shared by every candidate
    assert np.all(X[:, :7] == X[0, :7])


def test_trials_at_both_sigmas(pk):
    # N = (200, 120) at eps 1e-3: sigma = 2 gives w = 4 on a 400 x 240 grid, sigma = 1.25 gives
    # w = ceil(3 / 0.6) + 1 = 6 on 250 x 150 (both 2^a 3^b 5^c already)
    row = dict(seed=5, type=2, dim=2, N=[200, 120], M=80000, kind="gauss", spread=0.2, eps=1e-3,
               prec=0, w=4, skew=1.0, heuristic=[3, 12, 16, 1, 1024, 256],
               trials=[[3, 12, 16, 1, 1024, 256, 2.0, 0.5], [3, 12, 16, 1, 1024, 256, 1.25, 0.25],
                       [3, 8, 8, 1, 256, 128, 0.125]])
    X, T = pk.features(row)
    assert np.allclose(T, [-1.0, -2.0, -3.0])
    assert [pk.trial_sigma(t) for t in row["trials"]] == [2.0, 1.25, 2.0]
    assert X[0, 3] == pytest.approx(4 / 16) and X[2, 3] == pytest.approx(4 / 16)
    assert X[1, 3] == pytest.approx(6 / 16)
    assert X[0, 4] == pytest.approx(math.log2(400 * 240) / 32, abs=1e-7)
    assert X[1, 4] == pytest.approx(math.log2(250 * 150) / 32, abs=1e-7)
    assert X[1, 5] == pytest.approx(math.log2(80000 / (250 * 150)) / 8, abs=1e-7)
    # the tiling features do not depend on sigma
    assert np.all(X[0, 6:] == X[1, 6:])
    # a problem whose sigma = 1.25 plan cannot reach eps in single precision gets no such trials
    assert pk.sigma125_width(2, [200, 120], 1e-5, 80000, 0) is None
