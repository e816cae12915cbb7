"""Plain FP64 CPU oracle for alm2map and its transpose (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never imports
or links it, and it imports nothing from the product package.

The arithmetic lives in ``sht_oracle.c`` (plain C, compiled with gcc, no FMA
contraction, no fast-math); this module builds it, loads it with ctypes and
marshals numpy arrays.  Each function follows the paper (Hupca et al.,
"Spherical harmonic transform with GPUs", sec. 2.1):

* ``lam``               -- lambda_lm(x) by Eq. pmm, Eq. pm1m and the recurrence
                           of Eq. assLegRec with exponent tracking (Algorithm 2).
* ``alm2map``           -- Eq. DeltaDef then Eq. Delta2map, ring by ring
                           (Algorithm 1), the ring sum as a literal DFT.
* ``map2alm_adjoint``   -- the literal real-linear transpose of ``alm2map``
                           (Eq. map2almDef without quadrature weights).
* ``map2alm``           -- the quadrature-weighted analysis sum
                           a_lm = sum_p w_p y_p lambda_lm e^{-i m phi_p} (Eq.
                           map2almDef with the integral's measure), written out
                           as the literal transpose applied to w * y, divided
                           by the transpose's factor 2 for m > 0.
* ``lam_spin2``         -- the spin-2 functions 2lambda_lm (orders m and -m)
                           from the scalar lambda_lm, lambda_{l-1,m} by two
                           spin raisings (an extension beyond the paper, for
                           the polarisation field; definitions in sht_oracle.c).
* ``alm2map_spin2``     -- Q + iU = -sum (E + iB) 2Y_lm over all m of both
                           signs, pixel by pixel of each ring.
* ``gl_grid``, ``healpix_grid`` -- ring geometry (Gauss-Legendre by Newton
                           iteration; HEALPix RING from Gorski et al. 2005).

Pins: every function is checked in ``tests/test_oracle_pins.py`` against
closed forms, invariants and independent library routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sht_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no contraction).  Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            Lg = ctypes.c_long
            D = ctypes.c_double
            lib.orc_gl_nodes.argtypes = [I, P, P]
            lib.orc_healpix_rings.argtypes = [I, P, P, P, P]
            lib.orc_lambda.argtypes = [I, I, D, D, I, P]
            lib.orc_alm2map.argtypes = [I, I, I, P, P, P, P, P, Lg, I, P, P, I, P, I]
            lib.orc_map2alm_adjoint.argtypes = [I, I, I, P, P, P, P, P, Lg, I, P, P, I, P, I]
            lib.orc_lambda_spin2.argtypes = [I, I, D, D, P, P]
            lib.orc_alm2map_spin2.argtypes = [I, I, I, P, P, P, P, P, Lg, I, P, P, P, P, I, P, I]
            for f in (lib.orc_gl_nodes, lib.orc_healpix_rings, lib.orc_lambda,
                      lib.orc_alm2map, lib.orc_map2alm_adjoint, lib.orc_lambda_spin2,
                      lib.orc_alm2map_spin2):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def nalm(lmax: int, mmax: int) -> int:
    return (mmax + 1) * (2 * lmax + 2 - mmax) // 2


def _finish(g: dict) -> dict:
    nphi = g["nphi"]
    ofs = np.zeros(len(nphi), dtype=np.int64)
    if len(nphi) > 1:
        ofs[1:] = np.cumsum(nphi[:-1].astype(np.int64))
    g["ofs"] = ofs
    g["npix"] = int(nphi.astype(np.int64).sum())
    g["nrings"] = len(nphi)
    return g


def gl_grid(nrings: int, nphi: int) -> dict:
    """Gauss-Legendre grid: nrings nodes (north to south), nphi equispaced pixels, phi0 = 0."""
    lib = _load()
    x = np.zeros(nrings)
    w = np.zeros(nrings)
    if lib.orc_gl_nodes(nrings, _p(x), _p(w)) != 0:
        raise ValueError("bad nrings")
    st = np.sqrt((1.0 - x) * (1.0 + x))
    return _finish({"kind": "gl", "x": x, "st": st, "w": w,
                    "nphi": np.full(nrings, nphi, dtype=np.int32),
                    "phi0": np.zeros(nrings)})


def healpix_grid(nside: int) -> dict:
    """HEALPix RING grid (Gorski et al. 2005): 4 nside - 1 rings, 12 nside^2 pixels."""
    lib = _load()
    nr = 4 * nside - 1
    z = np.zeros(nr)
    st = np.zeros(nr)
    nphi = np.zeros(nr, dtype=np.int32)
    phi0 = np.zeros(nr)
    if lib.orc_healpix_rings(nside, _p(z), _p(st), _p(nphi), _p(phi0)) != 0:
        raise ValueError("bad nside")
    return _finish({"kind": "healpix", "x": z, "st": st, "nphi": nphi, "phi0": phi0})


def rings_grid(theta, nphi, phi0) -> dict:
    """A generic iso-latitude ring grid given by its colatitudes, lengths and first azimuths."""
    theta = np.asarray(theta, dtype=np.float64)
    return _finish({"kind": "rings", "x": np.cos(theta), "st": np.sin(theta),
                    "nphi": np.asarray(nphi, dtype=np.int32),
                    "phi0": np.asarray(phi0, dtype=np.float64)})


def lam(lmax: int, mmax: int, x: float, s: float | None = None, track: bool = True) -> np.ndarray:
    """lambda_lm(x) for all (l, m), m-major packed (length nalm)."""
    lib = _load()
    if s is None:
        s = float(np.sqrt((1.0 - x) * (1.0 + x)))
    out = np.zeros(nalm(lmax, mmax))
    if lib.orc_lambda(lmax, mmax, float(x), float(s), 1 if track else 0, _p(out)) != 0:
        raise ValueError("bad lmax/mmax")
    return out


def alm2map(grid: dict, lmax: int, mmax: int, alm: np.ndarray, rings=None,
            nthreads: int = 0, return_threads: bool = False):
    """alm2map of (nmaps, nalm) complex coefficients on ``grid``.

    Only the pixels of ``rings`` (default: all) are computed; the others are NaN.
    """
    lib = _load()
    alm = np.ascontiguousarray(np.atleast_2d(alm), dtype=np.complex128)
    nmaps = alm.shape[0]
    if alm.shape[1] != nalm(lmax, mmax):
        raise ValueError("alm has the wrong length")
    sel = np.arange(grid["nrings"], dtype=np.int32) if rings is None else \
        np.ascontiguousarray(rings, dtype=np.int32)
    out = np.full((nmaps, grid["npix"]), np.nan)
    x = np.ascontiguousarray(grid["x"], dtype=np.float64)
    st = np.ascontiguousarray(grid["st"], dtype=np.float64)
    phi0 = np.ascontiguousarray(grid["phi0"], dtype=np.float64)
    nphi = np.ascontiguousarray(grid["nphi"], dtype=np.int32)
    ofs = np.ascontiguousarray(grid["ofs"], dtype=np.int64)
    nt = lib.orc_alm2map(lmax, mmax, grid["nrings"], _p(x), _p(st), _p(phi0), _p(nphi),
                         _p(ofs), grid["npix"], nmaps, _p(alm), _p(out), len(sel), _p(sel),
                         int(nthreads))
    if nt < 0:
        raise RuntimeError("orc_alm2map failed (%d)" % nt)
    return (out, nt) if return_threads else out


def map2alm_adjoint(grid: dict, lmax: int, mmax: int, maps: np.ndarray, ms=None,
                    nthreads: int = 0) -> np.ndarray:
    """Real-linear transpose of alm2map; coefficients of m not in ``ms`` are NaN."""
    lib = _load()
    maps = np.ascontiguousarray(np.atleast_2d(maps), dtype=np.float64)
    nmaps = maps.shape[0]
    if maps.shape[1] != grid["npix"]:
        raise ValueError("map has the wrong length")
    sel = np.arange(mmax + 1, dtype=np.int32) if ms is None else \
        np.ascontiguousarray(ms, dtype=np.int32)
    out = np.full((nmaps, nalm(lmax, mmax)), np.nan + 0j, dtype=np.complex128)
    x = np.ascontiguousarray(grid["x"], dtype=np.float64)
    st = np.ascontiguousarray(grid["st"], dtype=np.float64)
    phi0 = np.ascontiguousarray(grid["phi0"], dtype=np.float64)
    nphi = np.ascontiguousarray(grid["nphi"], dtype=np.int32)
    ofs = np.ascontiguousarray(grid["ofs"], dtype=np.int64)
    nt = lib.orc_map2alm_adjoint(lmax, mmax, grid["nrings"], _p(x), _p(st), _p(phi0),
                                 _p(nphi), _p(ofs), grid["npix"], nmaps, _p(maps), _p(out),
                                 len(sel), _p(sel), int(nthreads))
    if nt < 0:
        raise RuntimeError("orc_map2alm_adjoint failed (%d)" % nt)
    return out


def pixel_weights(grid: dict) -> np.ndarray:
    """Quadrature weight of each ring's pixels: the Gauss weight x 2 pi / nphi on
    a Gauss-Legendre grid, the equal pixel area 4 pi / npix on HEALPix."""
    if grid["kind"] == "gl":
        return grid["w"] * (2.0 * np.pi / grid["nphi"])
    if grid["kind"] == "healpix":
        return np.full(grid["nrings"], 4.0 * np.pi / grid["npix"])
    raise ValueError("no quadrature weights for a generic ring grid")


def map2alm(grid: dict, lmax: int, mmax: int, maps: np.ndarray, weights=None) -> np.ndarray:
    """a_lm = sum_p w_p y_p lambda_lm(theta_p) e^{-i m phi_p}, m >= 0 (ring weights
    ``weights`` or the grid's own)."""
    w = pixel_weights(grid) if weights is None else np.asarray(weights, dtype=np.float64)
    maps = np.atleast_2d(np.asarray(maps, dtype=np.float64))
    wp = np.repeat(w, grid["nphi"].astype(np.int64))
    g = map2alm_adjoint(grid, lmax, mmax, maps * wp[None, :])
    m_of = np.concatenate([np.full(lmax + 1 - m, m) for m in range(mmax + 1)])
    g[:, m_of > 0] *= 0.5
    return g


def lam_spin2(lmax: int, mmax: int, x: float, s: float | None = None):
    """(plus, minus): 2lambda_lm(x) for orders m and -m, m-major packed (l < 2: 0)."""
    lib = _load()
    if s is None:
        s = float(np.sqrt((1.0 - x) * (1.0 + x)))
    plus = np.zeros(nalm(lmax, mmax))
    minus = np.zeros(nalm(lmax, mmax))
    if lib.orc_lambda_spin2(lmax, mmax, float(x), float(s), _p(plus), _p(minus)) != 0:
        raise ValueError("bad lmax/mmax or sin(theta) <= 0")
    return plus, minus


def alm2map_spin2(grid: dict, lmax: int, mmax: int, elm: np.ndarray, blm: np.ndarray, rings=None,
                  nthreads: int = 0):
    """(Q, U) maps of (nmaps, nalm) complex E and B coefficients; pixels of
    rings not selected are NaN."""
    lib = _load()
    elm = np.ascontiguousarray(np.atleast_2d(elm), dtype=np.complex128)
    blm = np.ascontiguousarray(np.atleast_2d(blm), dtype=np.complex128)
    nmaps = elm.shape[0]
    if elm.shape != blm.shape or elm.shape[1] != nalm(lmax, mmax):
        raise ValueError("E and B need shape (nmaps, nalm)")
    sel = np.arange(grid["nrings"], dtype=np.int32) if rings is None else \
        np.ascontiguousarray(rings, dtype=np.int32)
    q = np.full((nmaps, grid["npix"]), np.nan)
    u = np.full((nmaps, grid["npix"]), np.nan)
    x = np.ascontiguousarray(grid["x"], dtype=np.float64)
    st = np.ascontiguousarray(grid["st"], dtype=np.float64)
    phi0 = np.ascontiguousarray(grid["phi0"], dtype=np.float64)
    nphi = np.ascontiguousarray(grid["nphi"], dtype=np.int32)
    ofs = np.ascontiguousarray(grid["ofs"], dtype=np.int64)
    nt = lib.orc_alm2map_spin2(lmax, mmax, grid["nrings"], _p(x), _p(st), _p(phi0), _p(nphi), _p(ofs),
                               grid["npix"], nmaps, _p(elm), _p(blm), _p(q), _p(u), len(sel), _p(sel),
                               int(nthreads))
    if nt < 0:
        raise RuntimeError("orc_alm2map_spin2 failed (%d)" % nt)
    return q, u
