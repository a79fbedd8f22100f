"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws numbers: it holds none of the FMM arithmetic, and both
the CUDA library's tests/benchmarks and the FP64 oracle consume what it makes.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of stream s under seed k is mix(key(k, s) + (i+1)*GAMMA),
turned into a double in [0,1) from its top 53 bits.  Being counter-based, a
sub-range of any stream can be regenerated without drawing the rest.

Workloads (sizes and distributions as stated for the paper's uses):
  * uniform_cube      positions U[0,1)^3
  * masses            U(0,1] (drawn as 1-U[0,1)) or equal
  * m2l_pairs         cell pairs of side 1, offsets uniform over the 316
                      integer vectors of [-3,3]^3 minus [-1,1]^3, 16 source
                      particles U(cell) of unit mass per pair
  * plummer           Plummer sphere, scale radius a, radii beyond rmax
                      redrawn, isotropic directions
  * blobs             mixture of Gaussian blobs plus a uniform background
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        base = np.array([(seed * 0x100000001B3 + stream * 0x3C6EF372FE94F82B) & 0xFFFFFFFFFFFFFFFF],
                        dtype=np.uint64)
        return _mix(base + GAMMA)[0]


def u01(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n doubles in [0,1): draws start..start+n-1 of (seed, stream)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = _mix(_key(seed, stream) + i * GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_cube(n: int, seed: int):
    """Positions uniform in the unit cube [0,1)^3 (three arrays)."""
    return u01(seed, 0, n), u01(seed, 1, n), u01(seed, 2, n)


def masses_open_unit(n: int, seed: int) -> np.ndarray:
    """Masses uniform in (0,1], drawn as 1 - U[0,1)."""
    return 1.0 - u01(seed, 3, n)


def masses_equal(n: int) -> np.ndarray:
    return np.full(n, 1.0 / n)


def well_separated_offsets() -> np.ndarray:
    """The 316 integer vectors of [-3,3]^3 that are not in [-1,1]^3, (316,3)."""
    r = np.arange(-3, 4)
    o = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    keep = np.abs(o).max(axis=1) >= 2
    return o[keep].astype(np.int64)


def m2l_pairs(npairs: int, seed: int, per_cell: int = 16):
    """Independent M2L cell pairs of side 1.

    Returns (offsets (3, npairs) float64, src (3, per_cell, npairs) positions
    relative to each source-cell centre, uniform in [-1/2,1/2)^3, q (per_cell,
    npairs) unit masses).  The M2L vector r = z_target - z_source is the
    integer offset itself."""
    offs = well_separated_offsets()
    pick = np.minimum((u01(seed, 10, npairs) * len(offs)).astype(np.int64), len(offs) - 1)
    r = offs[pick].T.astype(np.float64).copy()
    src = np.stack([u01(seed, 11 + d, per_cell * npairs).reshape(per_cell, npairs) - 0.5
                    for d in range(3)])
    q = np.ones((per_cell, npairs))
    return r, src, q


def random_coefficients(ncoef: int, n: int, seed: int, stream: int = 20) -> np.ndarray:
    """Coefficient arrays [ncoef][n] with entries uniform in [-1,1)."""
    return (2.0 * u01(seed, stream, ncoef * n) - 1.0).reshape(ncoef, n)


def plummer(n: int, seed: int, a: float = 1.0, rmax: float = 20.0):
    """Plummer sphere: r = a / sqrt(U^(-2/3) - 1), radii > rmax redrawn,
    isotropic directions.  Returns x, y, z (centred at the origin)."""
    rad = np.empty(n)
    todo = np.arange(n)
    attempt = 0
    while len(todo):
        u = u01(seed, 30 + 3 * attempt, len(todo))
        u = np.where(u <= 0.0, 1e-300, u)
        with np.errstate(divide="ignore", invalid="ignore"):
            r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        ok = np.isfinite(r) & (r <= rmax)
        rad[todo[ok]] = r[ok]
        todo = todo[~ok]
        attempt += 1
    cth = 2.0 * u01(seed, 4, n) - 1.0
    phi = 2.0 * np.pi * u01(seed, 5, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return rad * sth * np.cos(phi), rad * sth * np.sin(phi), rad * cth


def blobs(n: int, seed: int, nblob: int = 32, background: float = 0.1,
          sigma_lo: float = 0.005, sigma_hi: float = 0.05):
    """Mixture of isotropic Gaussian blobs (centres U[0,1)^3, sigma U[lo,hi])
    holding (1-background) of the points in equal shares, plus a uniform
    background; points falling outside the unit cube are redrawn."""
    nb = int(round(n * background))
    ncl = n - nb
    cen = np.stack([u01(seed, 40 + d, nblob) for d in range(3)], 1)
    sig = sigma_lo + (sigma_hi - sigma_lo) * u01(seed, 43, nblob)
    which = np.arange(ncl) % nblob
    pos = np.empty((ncl, 3))
    todo = np.arange(ncl)
    attempt = 0
    while len(todo):
        m = len(todo)
        u1 = u01(seed, 50 + 4 * attempt, 2 * m).reshape(2, m)
        u2 = u01(seed, 51 + 4 * attempt, 2 * m).reshape(2, m)
        # Box-Muller: two pairs of uniforms give four normals, three used.
        r1 = np.sqrt(-2.0 * np.log(np.maximum(u1[0], 1e-300)))
        r2 = np.sqrt(-2.0 * np.log(np.maximum(u2[0], 1e-300)))
        g = np.stack([r1 * np.cos(2 * np.pi * u1[1]), r1 * np.sin(2 * np.pi * u1[1]),
                      r2 * np.cos(2 * np.pi * u2[1])], 1)
        w = which[todo]
        p = cen[w] + sig[w, None] * g
        ok = np.all((p >= 0.0) & (p < 1.0), axis=1)
        pos[todo[ok]] = p[ok]
        todo = todo[~ok]
        attempt += 1
    bx, by, bz = u01(seed, 60, nb), u01(seed, 61, nb), u01(seed, 62, nb)
    x = np.concatenate([pos[:, 0], bx])
    y = np.concatenate([pos[:, 1], by])
    z = np.concatenate([pos[:, 2], bz])
    perm = np.argsort(u01(seed, 63, n), kind="stable")
    return x[perm], y[perm], z[perm]
