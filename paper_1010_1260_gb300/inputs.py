"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and lays them out; it holds none of the
transform's arithmetic and imports nothing else from this package, so the
CPU oracle and the CUDA library can both be fed from it without sharing code.

Coefficient layout (m-major packed, the library's convention):
    idx(l, m) = m (2 lmax + 3 - m) / 2 + (l - m),   0 <= m <= mmax, m <= l <= lmax.

Workloads (the paper simulates a CMB sky, sec. 1 / Fig. 1; a Gaussian field with
power spectrum C_l = 1/(l(l+1)) stands in for it):
  * ``white``: Re, Im ~ N(0, 1/2) for m > 0 and a_l0 ~ N(0, 1) real.
  * ``cl``   : a_00 = a_1m = 0; for l >= 2, a_l0 ~ N(0, C_l) real and
               Re, Im ~ N(0, C_l / 2) for m > 0, with C_l = 1 / (l (l + 1)).
"""
from __future__ import annotations

import numpy as np


def nalm(lmax: int, mmax: int) -> int:
    """Number of stored (l, m) pairs, 0 <= m <= mmax, m <= l <= lmax."""
    return (mmax + 1) * (2 * lmax + 2 - mmax) // 2


def lm_arrays(lmax: int, mmax: int):
    """(l, m) of every packed index, as two int64 arrays of length nalm."""
    ls = []
    ms = []
    for m in range(mmax + 1):
        ls.append(np.arange(m, lmax + 1, dtype=np.int64))
        ms.append(np.full(lmax + 1 - m, m, dtype=np.int64))
    if not ls:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(ls), np.concatenate(ms)


def alm_index(l: int, m: int, lmax: int) -> int:
    return m * (2 * lmax + 3 - m) // 2 + (l - m)


def gaussian_alm(lmax: int, mmax: int, seed, nmaps: int = 1, spectrum: str = "cl") -> np.ndarray:
    """(nmaps, nalm) complex128 coefficients drawn from ``default_rng(seed)``.

    ``seed`` may be an int or a sequence (e.g. (3, b) for map b of a batch).
    """
    rng = np.random.default_rng(seed)
    ls, ms = lm_arrays(lmax, mmax)
    n = len(ls)
    out = np.zeros((nmaps, n), dtype=np.complex128)
    if spectrum == "white":
        var = np.ones(n)
    elif spectrum == "cl":
        var = np.zeros(n)
        ok = ls >= 2
        var[ok] = 1.0 / (ls[ok] * (ls[ok] + 1.0))
    else:
        raise ValueError(spectrum)
    m0 = ms == 0
    for b in range(nmaps):
        re = rng.standard_normal(n)
        im = rng.standard_normal(n)
        sd = np.where(m0, np.sqrt(var), np.sqrt(var / 2.0))
        out[b] = sd * re + 1j * np.where(m0, 0.0, sd * im)
    return out


def batch_alm(lmax: int, mmax: int, seed: int, nmaps: int, spectrum: str = "cl") -> np.ndarray:
    """Map b of the batch is drawn from seed (seed, b): the batch is a stack of singles."""
    return np.concatenate([gaussian_alm(lmax, mmax, (seed, b), 1, spectrum) for b in range(nmaps)])


def loss_weights(npix: int, seed, nmaps: int = 1):
    """w_p ~ U(0.5, 1.5) and d_p ~ N(0, 1), each (nmaps, npix) float64."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, size=(nmaps, npix))
    d = rng.standard_normal((nmaps, npix))
    return w, d


def gaussian_map(npix: int, seed, nmaps: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nmaps, npix))


def request_lmax(nreq: int, seed: int, lo: int = 64, hi: int = 2048) -> np.ndarray:
    """lmax log-uniform in [lo, hi], rounded to the nearest integer."""
    rng = np.random.default_rng(seed)
    v = np.exp(rng.uniform(np.log(lo), np.log(hi), size=nreq))
    return np.clip(np.rint(v).astype(np.int64), lo, hi)


def sample_rings(nrings: int, count: int, seed: int) -> np.ndarray:
    """A sorted, seeded subset of ring indices that always holds the first ring,
    the last ring and the middle (equator) ring."""
    rng = np.random.default_rng(seed)
    must = {0, nrings - 1, nrings // 2}
    rest = rng.choice(nrings, size=min(nrings, count), replace=False)
    sel = set(r for r in must if 0 <= r < nrings)
    for r in rest:
        if len(sel) >= count:
            break
        sel.add(int(r))
    return np.asarray(sorted(sel), dtype=np.int32)


def _largest_prime_factor(n: int) -> int:
    best, p = 1, 2
    while p * p <= n:
        while n % p == 0:
            best, n = p, n // p
        p += 1
    return max(best, n) if n > 1 else best


def healpix_ring_sample(nside: int, count: int, seed: int, large_prime: int = 29, n_large: int = 12,
                        n_smooth_cap: int = 12):
    """A seeded, sorted sample of HEALPix RING-scheme ring indices stratified by
    ring class: both polar rings, the equator, ``n_large`` polar-cap rings whose
    length 4 i has a prime factor >= ``large_prime``, ``n_smooth_cap`` cap rings
    whose length has none, and equatorial-belt rings for the rest.  Returns
    (rings, classes) with classes[r] one of "pole", "equator", "cap_large_prime",
    "cap_smooth", "belt"."""
    nrings = 4 * nside - 1
    rng = np.random.default_rng(seed)

    def cap_i(r):  # ring index -> i of the Gorski numbering (1 .. 2 nside), or None in the belt
        i = r + 1 if r < 2 * nside else nrings - r
        return i if i < nside else None

    cls = {}
    cls[0] = cls[nrings - 1] = "pole"
    cls[nrings // 2] = "equator"
    caps_large = [r for r in range(nrings) if r not in cls and cap_i(r) is not None
                  and _largest_prime_factor(cap_i(r)) >= large_prime]
    caps_smooth = [r for r in range(nrings) if r not in cls and cap_i(r) is not None
                   and _largest_prime_factor(cap_i(r)) < large_prime]
    belt = [r for r in range(nrings) if r not in cls and cap_i(r) is None]
    for pool, k, name in ((caps_large, n_large, "cap_large_prime"), (caps_smooth, n_smooth_cap, "cap_smooth")):
        for r in rng.choice(pool, size=min(k, len(pool)), replace=False) if pool else []:
            cls[int(r)] = name
    rest = max(0, count - len(cls))
    for r in rng.choice(belt, size=min(rest, len(belt)), replace=False) if belt else []:
        cls[int(r)] = "belt"
    rings = np.asarray(sorted(cls), dtype=np.int32)
    return rings, {int(r): cls[int(r)] for r in rings}
