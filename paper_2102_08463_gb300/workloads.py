"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers; it holds none of the transform's
arithmetic.  Every draw comes from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): state_i = seed +
(i+1) * 0x9E3779B97F4A7C15, then the published three-step mixer.  Uniform
doubles take the top 53 bits; normals use Box-Muller on two uniform streams.

Point distributions follow the paper's test setup (Sec. 5): "rand" is i.i.d.
uniform on [-pi, pi)^d, "cluster" is i.i.d. uniform on the box [0, 8 h]^d with h the
fine-grid spacing.  "gauss" is the wrapped normal N(0, s^2) per coordinate used
by the clustered 3D workload.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

BASE_SEED = 2102084630


def splitmix64(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """`count` outputs of SplitMix64 started at seed + stream * 2^40 (uint64)."""
    with np.errstate(over="ignore"):
        s0 = np.uint64((int(seed) + (int(stream) << 40)) & 0xFFFFFFFFFFFFFFFF)
        z = s0 + (np.arange(1, count + 1, dtype=np.uint64) * _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, count, stream) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller."""
    u1 = uniform01(seed, count, 2 * stream + 1000)
    u2 = uniform01(seed, count, 2 * stream + 1001)
    r = np.sqrt(-2.0 * np.log1p(-u1))
    return r * np.cos(2.0 * math.pi * u2)


def points(kind: str, dim: int, M: int, seed: int, dtype=np.float32, n=None,
           spread: float = 0.05 * math.pi):
    """List of `dim` coordinate arrays of M points in the plan's precision.

    kind: "rand" (uniform on [-pi, pi)), "gauss" (wrapped N(0, spread^2)),
    "cluster" (uniform on [0, 8 h_i], needs the fine-grid sizes n), "mixture"
    (8 equally likely wrapped Gaussians N(c_k, spread^2), centres uniform).
    """
    out = []
    if kind == "mixture":
        comp = np.minimum((uniform01(seed, M, stream=90) * 8).astype(np.int64), 7)
        for d in range(dim):
            centres = -math.pi + 2.0 * math.pi * uniform01(seed, 8, stream=91 + d)
            g = centres[comp] + spread * normal(seed, M, stream=95 + d)
            x = g - 2.0 * math.pi * np.floor((g + math.pi) / (2.0 * math.pi))
            out.append(np.ascontiguousarray(x.astype(dtype)))
        return out
    for d in range(dim):
        if kind == "rand":
            x = -math.pi + 2.0 * math.pi * uniform01(seed, M, stream=d)
        elif kind == "gauss":
            g = spread * normal(seed, M, stream=d)
            x = g - 2.0 * math.pi * np.floor((g + math.pi) / (2.0 * math.pi))
        elif kind == "cluster":
            if n is None:
                raise ValueError("cluster points need the fine-grid sizes n")
            h = 2.0 * math.pi / n[d]
            x = 8.0 * h * uniform01(seed, M, stream=d)
        else:
            raise ValueError("unknown point distribution %r" % kind)
        out.append(np.ascontiguousarray(x.astype(dtype)))
    return out


def strengths(M: int, seed: int, dtype=np.complex64, ntransf: int = 1) -> np.ndarray:
    """Complex strengths with re and im i.i.d. N(0, 1); shape (ntransf, M) or (M,)."""
    re = normal(seed, M * ntransf, stream=20)
    im = normal(seed, M * ntransf, stream=21)
    c = (re + 1j * im).astype(dtype)
    return c.reshape(ntransf, M) if ntransf > 1 else c


def modes(N, seed: int, dtype=np.complex64, ntransf: int = 1) -> np.ndarray:
    """Fourier coefficients f with re and im i.i.d. N(0, 1), shape ([ntransf,] N3, N2, N1)."""
    shape = tuple(reversed(tuple(int(v) for v in N)))
    cnt = int(np.prod(shape)) * ntransf
    re = normal(seed, cnt, stream=30)
    im = normal(seed, cnt, stream=31)
    f = (re + 1j * im).astype(dtype)
    return f.reshape((ntransf,) + shape) if ntransf > 1 else f.reshape(shape)


def sample_indices(total: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct indices in [0, total), sorted (for sampled oracle checks)."""
    count = min(count, total)
    keys = splitmix64(seed, total, stream=40) if total <= 50_000_000 else None
    if keys is not None:
        return np.sort(np.argsort(keys, kind="stable")[:count]).astype(np.int64)
    picks = set()
    u = uniform01(seed, 4 * count, stream=41)
    for v in u:
        picks.add(int(v * total))
        if len(picks) == count:
            break
    return np.asarray(sorted(picks), dtype=np.int64)
