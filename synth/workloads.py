"""Workload presets and the seeded draws of the batched and served mixes.

The presets are the benchmark problems: two-species (proton/neutron)
nuclei in an HO basis with total 2M = 0, an optional Nmax cut on the excess
HO quanta, and seeded TBMEs (see ``tbme``).

* ``c0``  4p+4n, shells N <= 1 (8 states per species), no Nmax cut, FP64.
* ``c1``  4p+4n, shells N <= 4 (70 states), Nmax = 4, FP32 H, block size 8.
* ``c2``  as c1 with Nmax = 6; ``c2_sub`` is its Nmax = 2 subspace.
* ``batch``: Z, N uniform on 2..6 and Nmax uniform on 0..4 in shells N <= 3
  (40 states), one TBME seed per problem; callers keep the draws whose
  dimension lies in [1e2, 1e5].
* ``serve``: Poisson arrivals of requests drawn from the batch mix plus 5 %
  c1-sized requests, each asking for 1..10 eigenvalues.
"""

from dataclasses import dataclass, replace

import numpy as np

from .tbme import splitmix64_mix


@dataclass(frozen=True)
class Preset:
    name: str
    n_shell_max: int
    Z: int
    N: int
    nmax: int          # -1: no truncation
    twoM: int = 0
    hbar_omega: float = 20.0
    seed: int = 0
    value_type: str = "f32"   # "f32", "f64" or "bf16" (bf16 values, f32 row scale)
    k: int = 5                # eigenvalues wanted
    block: int = 8            # Lanczos / SpMM block size


PRESETS = {
    "c0": Preset("c0", 1, 4, 4, -1, seed=0, value_type="f64", k=5),
    "c1": Preset("c1", 4, 4, 4, 4, seed=1, value_type="f32", k=5),
    "c2": Preset("c2", 4, 4, 4, 6, seed=2, value_type="f32", k=10),
    "c2_sub": Preset("c2_sub", 4, 4, 4, 2, seed=2, value_type="f32", k=10),
}


def preset(name, **changes):
    """Return a preset, optionally with fields replaced."""
    p = PRESETS[name]
    return replace(p, **changes) if changes else p


def _uniform_stream(seed, n, stream):
    """n uniforms in [0, 1) from SplitMix64 positions of (seed, stream)."""
    gamma = np.uint64(0x9E3779B97F4A7C15)
    pos = (np.uint64(stream) << np.uint64(40)) + np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = splitmix64_mix(np.uint64(seed) + pos * gamma)
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def batch_candidates(seed=3, count=4096):
    """Candidate draws (Z, N, nmax, tbme_seed) of the batched mix, in order.

    Z and N are uniform on 2..6, nmax uniform on 0..4, shells N <= 3.  The
    caller filters them by basis dimension.
    """
    u = _uniform_stream(seed, 3 * count, 0).reshape(count, 3)
    Z = 2 + np.floor(u[:, 0] * 5).astype(int)
    N = 2 + np.floor(u[:, 1] * 5).astype(int)
    nmax = np.floor(u[:, 2] * 5).astype(int)
    return [dict(n_shell_max=3, Z=int(Z[i]), N=int(N[i]), nmax=int(nmax[i]),
                 seed=int(1000 * seed + i), k=5) for i in range(count)]


def serve_requests(rate_per_s, n_requests, seed=4, big_fraction=0.05,
                   small_pool=None):
    """A Poisson request stream.

    Returns a list of dicts with ``t_arrival`` (s, from 0), the problem fields
    and ``k`` (1..10).  ``small_pool`` is the list of accepted batch-mix draws
    to sample the small requests from; big requests are c1-sized.
    """
    if small_pool is None or len(small_pool) == 0:
        raise ValueError("serve_requests needs the accepted batch-mix pool")
    u = _uniform_stream(seed, 4 * n_requests, 1).reshape(n_requests, 4)
    gaps = -np.log1p(-u[:, 0]) / rate_per_s
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n_requests):
        k = 1 + int(np.floor(u[i, 3] * 10))
        if u[i, 1] < big_fraction:
            p = PRESETS["c1"]
            req = dict(n_shell_max=p.n_shell_max, Z=p.Z, N=p.N, nmax=p.nmax)
        else:
            req = dict(small_pool[int(np.floor(u[i, 2] * len(small_pool)))])
            req.pop("k", None)
        req["seed"] = int(100000 * seed + i)
        req["k"] = k
        req["t_arrival"] = float(t[i])
        out.append(req)
    return out

