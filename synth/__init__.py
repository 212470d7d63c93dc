"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module draws random numbers and nothing else: grid sizes, per-element
coefficients, nodal loads and per-subdomain moduli.  It holds none of the
preconditioner's arithmetic (no assembly, no partition, no factorisation), so
both the CPU oracle and the CUDA path can consume its arrays without sharing
any of the method's code.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used counter-style: the i-th draw of stream `seed`
is mix64(seed + (i + 1) * 0x9E3779B97F4A7C15).  Normals come from Box-Muller.

The workloads follow the 3-D configurations the method is measured on (Sec. 4
generalised to 3-D per its conclusions): a unit cube meshed by n^3 nodes with
trilinear hexahedra, homogeneous Dirichlet on the whole boundary.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` SplitMix64 outputs (uint64) of stream `seed`, starting at draw `offset`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each draw times 2^-53."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, count)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller; draw pairs (2k, 2k+1) give output k."""
    u = uniform01(seed, 2 * count)
    u1 = 1.0 - u[0::2]            # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def randint(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform on {lo, ..., hi} (inclusive), by multiply-shift of 32 high bits."""
    span = np.uint64(hi - lo + 1)
    top = splitmix64(seed, count) >> np.uint64(32)
    return (lo + ((top * span) >> np.uint64(32))).astype(np.int64)


# ----------------------------------------------------------------------------
# Workloads.  n = nodes per side (including the two Dirichlet boundary layers),
# so a problem has (n-2)^3 interior nodes and (n-1)^3 elements.
# ----------------------------------------------------------------------------

def n_elements(n: int) -> int:
    return (n - 1) ** 3


def n_interior(n: int) -> int:
    return (n - 2) ** 3


def poisson_const(n: int, depth: int, f_seed: int) -> dict:
    """Constant-coefficient Poisson: kappa = 1, nodal f ~ U[-1, 1]."""
    return dict(n=n, depth=depth, kappa=np.ones(n_elements(n)),
                f=uniform(f_seed, n_interior(n)))


def diffusion_lognormal(n: int, depth: int, kappa_seed: int, f_seed: int,
                        sigma: float = 1.0) -> dict:
    """kappa_e = exp(sigma * z_e), z_e iid N(0, 1) per element; nodal f ~ U[-1, 1]."""
    return dict(n=n, depth=depth,
                kappa=np.exp(sigma * normal(kappa_seed, n_elements(n))),
                f=uniform(f_seed, n_interior(n)))


def batched_sizes(count: int, seed: int, lo: int = 17, hi: int = 65) -> np.ndarray:
    """Grid sides n_p ~ U{lo..hi} for a batch of independent problems."""
    return randint(seed, count, lo, hi)


def batched_depth(n: int) -> int:
    """8 subdomains for small problems, 64 for the rest (n - 1 < 32 -> depth 1)."""
    return 1 if n - 1 < 32 else 2


def batched_poisson(count: int, size_seed: int, f_seed0: int,
                    lo: int = 17, hi: int = 65) -> list[dict]:
    sizes = batched_sizes(count, size_seed, lo, hi)
    return [poisson_const(int(n), batched_depth(int(n)), f_seed0 + p)
            for p, n in enumerate(sizes)]


def gaussian_field(n: int, seed: int, corr: float = 0.1) -> np.ndarray:
    """Per-element Gaussian random field: iid N(0,1) smoothed by a separable
    Gaussian kernel of standard deviation `corr` (unit-cube lengths), truncated at
    3 sigma, rescaled to unit sample variance.  Returned flat, element order
    ex + (n-1)*(ey + (n-1)*ez)."""
    ne = n - 1
    z = normal(seed, ne ** 3).reshape(ne, ne, ne)        # [ez, ey, ex]
    s = corr * ne                                          # std in elements
    r = int(np.ceil(3.0 * s))
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / s) ** 2)
    k /= k.sum()
    for axis in range(3):
        z = np.apply_along_axis(lambda v: np.convolve(v, k, mode="same"), axis, z)
    z = (z - z.mean()) / z.std()
    return z.reshape(-1)


def elasticity_moduli(n_leaves: int, seed: int) -> np.ndarray:
    """Young's modulus per leaf subdomain, log-uniform on [1, 1e3]."""
    return 10.0 ** uniform(seed, n_leaves, 0.0, 3.0)


# The five measured workloads (sizes and seeds of the 3-D configurations).
WORKLOADS = {
    "poisson13": dict(kind="poisson", n=13, depth=1, f_seed=1),
    "diffusion129": dict(kind="lognormal", n=129, depth=3, kappa_seed=2, f_seed=3),
    "batched256": dict(kind="batched", count=256, size_seed=4, f_seed0=5),
    "adjoint65": dict(kind="grf", n=65, depth=2, m_seed=6, f_seed=7, m2_seed=8),
    "elasticity97": dict(kind="elasticity", n=97, depth=4, e_seed=9, f_seed=10),
}


def make(name: str, n: int | None = None, depth: int | None = None) -> dict:
    """Build a scalar workload by name; `n`/`depth` override the size for scaled samples."""
    w = dict(WORKLOADS[name])
    if n is not None:
        w["n"] = n
    if depth is not None:
        w["depth"] = depth
    if w["kind"] == "poisson":
        return poisson_const(w["n"], w["depth"], w["f_seed"])
    if w["kind"] == "lognormal":
        return diffusion_lognormal(w["n"], w["depth"], w["kappa_seed"], w["f_seed"])
    raise ValueError(f"workload {name} is not a single scalar problem")
