"""Seeded synthetic inputs for HENN workloads.

This module only draws random inputs (base points, queries, per-query beam
widths).  It holds none of the index's arithmetic and is imported by both the
FP64 oracle's tests and the CUDA path's tests and benchmark, so the two sides
see identical inputs.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) evaluated counter-style in numpy, so a value
depends only on (seed, tag, counter) and never on chunking or platform.
Uniforms take the top 53 bits; normals use the Box-Muller transform in FP64;
every dataset is cast to float32 at the end.

Workloads (the paper evaluates on SIFT/GloVe/MNIST and on exponential
synthetic data, Sec. 4 and App. G; none of those files are used here, these
generators stand in for them):
  * uniform_cube      : i.i.d. U[0,1)^d
  * gaussian_mixture  : isotropic clusters, centres N(0,I), per-cluster sigma
                        U[0.1,0.5]; optional affine rescale to [0,255]
                        (SIFT-like range) or unit-length normalisation
  * nested_shells     : points uniform on spheres of radius 2^-i
  * exponential       : i.i.d. Exp(lambda) coordinates (App. G, "Methods and
                        Datasets")
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "splitmix64",
    "uniform_stream",
    "normal_stream",
    "uniform_cube",
    "gaussian_mixture",
    "nested_shells",
    "shell_queries",
    "exponential",
    "log_uniform_int",
    "workload",
    "WORKLOADS",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22  # values per chunk when streaming large arrays


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, tag: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        h = _mix(s + _GAMMA)
        h = _mix(h ^ (np.uint64(tag & 0xFFFFFFFFFFFFFFFF) * _GAMMA + _GAMMA))
    return h[0]


def splitmix64(state: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+count-1 of SplitMix64 seeded with `state`."""
    with np.errstate(over="ignore"):
        j = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(np.uint64(state & 0xFFFFFFFFFFFFFFFF) + j * _GAMMA)


def _raw(seed: int, tag: int, count: int, start: int = 0) -> np.ndarray:
    return splitmix64(int(_key(seed, tag)), count, start)


def uniform_stream(seed: int, tag: int, count: int, start: int = 0, open0: bool = False) -> np.ndarray:
    """FP64 uniforms in [0,1) (or (0,1] with open0=True) from stream (seed, tag)."""
    u = _raw(seed, tag, count, start) >> np.uint64(11)
    if open0:
        u = u + np.uint64(1)
    return u.astype(np.float64) * (1.0 / 9007199254740992.0)


def normal_stream(seed: int, tag: int, count: int, start: int = 0) -> np.ndarray:
    """FP64 standard normals (Box-Muller, cosine branch) from stream (seed, tag)."""
    u1 = uniform_stream(seed, 2 * tag + 1, count, start, open0=True)
    u2 = uniform_stream(seed, 2 * tag + 2, count, start)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _bounded(seed: int, tag: int, count: int, bound: int, start: int = 0) -> np.ndarray:
    """Integers uniform in [0, bound) via 64x64 multiply-high (Lemire)."""
    u = _raw(seed, tag, count, start)
    hi = u >> np.uint64(32)
    lo = u & np.uint64(0xFFFFFFFF)
    b = np.uint64(bound)
    # (u * bound) >> 64 for bound < 2^32, split to stay in 64-bit lanes
    t = lo * b
    t = (hi * b) + (t >> np.uint64(32))
    return (t >> np.uint64(32)).astype(np.int64)


def uniform_cube(n: int, d: int, seed: int) -> np.ndarray:
    """n points i.i.d. uniform in [0,1)^d, float32."""
    out = np.empty((n, d), dtype=np.float32)
    rows = max(1, _CHUNK // d)
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        out[r0:r1] = uniform_stream(seed, 11, (r1 - r0) * d, r0 * d).reshape(r1 - r0, d)
    return out


def _mixture_params(d: int, n_clusters: int, mixture_seed: int):
    centres = normal_stream(mixture_seed, 21, n_clusters * d).reshape(n_clusters, d)
    sigma = 0.1 + 0.4 * uniform_stream(mixture_seed, 22, n_clusters)
    return centres, sigma


def gaussian_mixture(
    n: int,
    d: int,
    n_clusters: int,
    seed: int,
    mixture_seed: int = 0,
    rescale_from: tuple[float, float] | None = None,
    rescale_to_255: bool = False,
    normalise: bool = False,
) -> tuple[np.ndarray, tuple[float, float] | None]:
    """Gaussian mixture: x = centre[c] + sigma[c] * N(0, I), c uniform.

    The mixture (centres, sigmas) is fixed by `mixture_seed`; the points by
    `seed`, so base points and queries share one mixture.  With
    rescale_to_255 the global min/max of *this* draw (or `rescale_from` when
    given, e.g. the base set's range for queries) is mapped affinely to
    [0, 255]; values are not clamped.  With normalise every vector is scaled
    to unit length.  Returns (points float32, (min, max) used or None).
    """
    centres, sigma = _mixture_params(d, n_clusters, mixture_seed)
    out = np.empty((n, d), dtype=np.float32)
    rows = max(1, _CHUNK // d)
    vmin, vmax = math.inf, -math.inf
    tmp = np.empty((n, d), dtype=np.float64) if (rescale_to_255 and rescale_from is None) else None
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        cid = _bounded(seed, 31, r1 - r0, n_clusters, r0)
        z = normal_stream(seed, 32, (r1 - r0) * d, r0 * d).reshape(r1 - r0, d)
        x = centres[cid] + sigma[cid, None] * z
        if normalise:
            x = x / np.linalg.norm(x, axis=1, keepdims=True)
        if tmp is not None:
            tmp[r0:r1] = x
            vmin = min(vmin, float(x.min()))
            vmax = max(vmax, float(x.max()))
        elif rescale_to_255:
            lo, hi = rescale_from
            out[r0:r1] = (x - lo) * (255.0 / (hi - lo))
        else:
            out[r0:r1] = x
    if tmp is not None:
        out[:] = (tmp - vmin) * (255.0 / (vmax - vmin))
        return out, (vmin, vmax)
    return out, (tuple(rescale_from) if rescale_from is not None else None)


def nested_shells(n_per_shell: int, n_shells: int, d: int, seed: int) -> np.ndarray:
    """Shell i (i = 0..n_shells-1) holds n_per_shell points radius 2^-i * g/|g|."""
    n = n_per_shell * n_shells
    out = np.empty((n, d), dtype=np.float32)
    rows = max(1, _CHUNK // d)
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        g = normal_stream(seed, 41, (r1 - r0) * d, r0 * d).reshape(r1 - r0, d)
        shell = np.arange(r0, r1) // n_per_shell
        radius = np.ldexp(1.0, -shell)
        out[r0:r1] = (g / np.linalg.norm(g, axis=1, keepdims=True)) * radius[:, None]
    return out


def shell_queries(nq: int, d: int, seed: int, r_lo_exp: int = -20, r_hi_exp: int = -18) -> np.ndarray:
    """Uniform directions, radius log-uniform in [2^r_lo_exp, 2^r_hi_exp]."""
    g = normal_stream(seed, 42, nq * d).reshape(nq, d)
    u = uniform_stream(seed, 43, nq)
    radius = np.exp2(r_lo_exp + (r_hi_exp - r_lo_exp) * u)
    return ((g / np.linalg.norm(g, axis=1, keepdims=True)) * radius[:, None]).astype(np.float32)


def exponential(n: int, d: int, lam: float, seed: int) -> np.ndarray:
    """Coordinates i.i.d. exponential with rate lam (mean 1/lam)."""
    out = np.empty((n, d), dtype=np.float32)
    rows = max(1, _CHUNK // d)
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        u = uniform_stream(seed, 51, (r1 - r0) * d, r0 * d, open0=True)
        out[r0:r1] = (-np.log(u) / lam).reshape(r1 - r0, d)
    return out


def log_uniform_int(count: int, lo: int, hi: int, seed: int, tag: int = 61) -> np.ndarray:
    """round(exp(U[ln lo, ln hi])) as int32 (per-query beam widths)."""
    u = uniform_stream(seed, tag, count)
    return np.rint(np.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u)).astype(np.int32)


# ---------------------------------------------------------------------------
# Named workloads.  Base seed 0, query seed 1.
# ---------------------------------------------------------------------------
WORKLOADS = {
    "uniform-10k-d32": dict(n=10_000, d=32, nq=1_000, k=10, metric="l2"),
    "mixture-1m-d128": dict(n=1_000_000, d=128, nq=10_000, k=10, metric="l2", clusters=1_000),
    "shells-1m-d64": dict(n=1_000_000, d=64, nq=10_000, k=10, metric="l2"),
    "mixture-1m-d960": dict(n=1_000_000, d=960, nq=10_000, k=10, metric="l2", clusters=500),
    "angular-10m-d96": dict(n=10_000_000, d=96, nq=10_000, k=10, metric="angular", clusters=10_000),
    # the paper's own synthetic data (App. G): i.i.d. exponential coordinates
    "exponential-50k-d32-l4": dict(n=50_000, d=32, nq=10_000, k=10, metric="l2", lam=4.0),
    "exponential-50k-d32-l32": dict(n=50_000, d=32, nq=10_000, k=10, metric="l2", lam=32.0),
    "exponential-50k-d32-l256": dict(n=50_000, d=32, nq=10_000, k=10, metric="l2", lam=256.0),
    "exponential-1m-d16-l4": dict(n=1 << 20, d=16, nq=10_000, k=10, metric="l2", lam=4.0),
    "exponential-1m-d32-l4": dict(n=1 << 20, d=32, nq=10_000, k=10, metric="l2", lam=4.0),
}


def workload(name: str, n: int | None = None, nq: int | None = None):
    """Return (base, queries, info) for a named workload.

    `n` / `nq` shrink the workload for tests (same generator, same mixture,
    first n points of the base stream).  For the SIFT-like mixture the
    [0,255] map is taken from the generated base set, queries reuse it.
    info carries per-query beam widths for the shells workload.
    """
    spec = dict(WORKLOADS[name])
    n = spec["n"] if n is None else n
    nq = spec["nq"] if nq is None else nq
    d = spec["d"]
    info = dict(spec, n=n, nq=nq, name=name)
    if name == "uniform-10k-d32":
        X = uniform_cube(n, d, seed=0)
        Q = uniform_cube(nq, d, seed=1)
    elif name == "mixture-1m-d128":
        X, rng = gaussian_mixture(n, d, spec["clusters"], seed=0, rescale_to_255=True)
        Q, _ = gaussian_mixture(nq, d, spec["clusters"], seed=1, rescale_from=rng, rescale_to_255=True)
    elif name == "shells-1m-d64":
        per = max(1, n // 20)
        X = nested_shells(per, 20, d, seed=0)
        Q = shell_queries(nq, d, seed=1)
        info["ef_per_query"] = log_uniform_int(nq, 32, 512, seed=1)
    elif name == "mixture-1m-d960":
        X, _ = gaussian_mixture(n, d, spec["clusters"], seed=0)
        Q, _ = gaussian_mixture(nq, d, spec["clusters"], seed=1)
    elif name == "angular-10m-d96":
        X, _ = gaussian_mixture(n, d, spec["clusters"], seed=0, normalise=True)
        Q, _ = gaussian_mixture(nq, d, spec["clusters"], seed=1, normalise=True)
    elif name.startswith("exponential-"):
        X = exponential(n, d, spec["lam"], seed=0)
        Q = exponential(nq, d, spec["lam"], seed=1)
    else:  # pragma: no cover
        raise KeyError(name)
    return X, Q, info
