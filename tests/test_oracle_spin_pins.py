"""Pins of the oracle's spin-2 (polarisation) synthesis, CPU only.

The spin-2 functions 2lambda_lm and the Q/U synthesis are pinned against
things other than the oracle's own formula:
  * closed forms: 2Y_lm = ð ð Y_lm / K_l and -2Y_lm = ð̄ ð̄ Y_lm / K_l taken
    symbolically by sympy from its own Y_lm, l <= 4, both signs of m, several
    colatitudes (the oracle instead eliminates the derivatives with the
    Legendre equation and the derivative recurrence);
  * the addition theorem of spin-weighted harmonics,
    sum_{|m|<=l} |2Y_lm|^2 = (2l+1)/(4 pi), to lmax 2048 including HEALPix
    polar rings;
  * orthonormality of 2Y_lm on the sphere by Gauss-Legendre quadrature;
  * the synthesis against a pixel-by-pixel sum of the sympy closed forms on a
    tiny HEALPix grid, and a Gauss-Legendre round trip (the quadrature
    analysis of the oracle's Q + iU returns E and B).
"""
import math

import numpy as np
import pytest

sympy = pytest.importorskip("sympy")


def _nalm(L, M):
    return (M + 1) * (2 * L + 2 - M) // 2


def _idx(l, m, L):
    return m * (2 * L + 3 - m) // 2 + (l - m)


def _sympy_spin2(lmax):
    """{(l, m): (f_plus(theta), f_minus(theta))} with 2Y_lm = f_plus e^{i m phi},
    -2Y_lm = f_minus e^{i m phi}, from sympy's Ynm by symbolic spin raisings."""
    th, ph = sympy.symbols("theta phi", real=True)
    st = sympy.sin(th)

    def eth(f, s):      # spin raising of a spin-s quantity
        return -(st ** s) * (sympy.diff(f * st ** (-s), th) + sympy.I / st * sympy.diff(f * st ** (-s), ph))

    def ethbar(f, s):   # spin lowering of a spin-s quantity
        return -(st ** (-s)) * (sympy.diff(f * st ** s, th) - sympy.I / st * sympy.diff(f * st ** s, ph))

    out = {}
    for l in range(2, lmax + 1):
        K = sympy.sqrt((l - 1) * l * (l + 1) * (l + 2))
        for m in range(-l, l + 1):
            Y = sympy.Ynm(l, m, th, ph).expand(func=True)
            p2 = sympy.simplify(eth(eth(Y, 0), 1) / K * sympy.exp(-sympy.I * m * ph))
            m2 = sympy.simplify(ethbar(ethbar(Y, 0), -1) / K * sympy.exp(-sympy.I * m * ph))
            out[(l, m)] = (sympy.lambdify(th, p2, "numpy"), sympy.lambdify(th, m2, "numpy"))
    return out


@pytest.fixture(scope="module")
def closed_forms():
    return _sympy_spin2(4)


@pytest.mark.parametrize("theta", [0.31, 0.9, 1.5707963267948966, 2.2, 3.0])
def test_spin2_closed_forms(oracle_mod, closed_forms, theta):
    L = 4
    plus, minus = oracle_mod.lam_spin2(L, L, math.cos(theta), math.sin(theta))
    for (l, m), (fp, fm) in closed_forms.items():
        am = abs(m)
        got = plus[_idx(l, am, L)] if m >= 0 else minus[_idx(l, am, L)]
        want = complex(fp(theta))
        assert abs(want.imag) < 1e-12
        assert abs(got - want.real) < 1e-12, (l, m, got, want)
        # -2lambda_lm = (-1)^m 2lambda_{l,-m}: the relation the GPU kernels use
        other = (minus[_idx(l, am, L)] if m >= 0 else plus[_idx(l, am, L)]) * (-1) ** am
        assert abs(other - complex(fm(theta)).real) < 1e-12, (l, m)


@pytest.mark.parametrize("x", [0.999999, 0.97, 0.5, 0.0, -0.3, -0.9999])
def test_spin2_addition_theorem(oracle_mod, x):
    L = 2048
    plus, minus = oracle_mod.lam_spin2(L, L, x)
    tot = np.zeros(L + 1)
    for m in range(L + 1):
        sl = slice(_idx(m, m, L), _idx(m, m, L) + L + 1 - m)
        tot[m:] += plus[sl] ** 2 + (minus[sl] ** 2 if m > 0 else 0.0)
    ls = np.arange(2, L + 1)
    want = (2 * ls + 1) / (4 * np.pi)
    assert np.max(np.abs(tot[2:] - want) / want) < 1e-9


def test_spin2_addition_theorem_healpix_polar_rings(oracle_mod):
    g = oracle_mod.healpix_grid(1024)
    L = 2048
    for r in (0, 1, 5, 4094):
        plus, minus = oracle_mod.lam_spin2(L, L, g["x"][r], g["st"][r])
        tot = np.zeros(L + 1)
        for m in range(L + 1):
            sl = slice(_idx(m, m, L), _idx(m, m, L) + L + 1 - m)
            tot[m:] += plus[sl] ** 2 + (minus[sl] ** 2 if m > 0 else 0.0)
        ls = np.arange(2, L + 1)
        want = (2 * ls + 1) / (4 * np.pi)
        # near the poles the two spin raisings cancel terms of size ~ l^2 / sin^2
        # (measured: 1.3e-11 at the second ring)
        assert np.max(np.abs(tot[2:] - want) / want) < 1e-9


def test_spin2_orthonormality_gauss_legendre(oracle_mod):
    L, n = 40, 42
    g = oracle_mod.gl_grid(n, 2 * L + 2)
    tabs = [oracle_mod.lam_spin2(L, L, g["x"][r], g["st"][r]) for r in range(n)]
    for m in (0, 1, 2, 5, 17, 40):
        ls = np.arange(max(2, m), L + 1)
        for sign in (0, 1):
            F = np.array([[t[sign][_idx(l, m, L)] for l in ls] for t in tabs])  # [ring, l]
            G = 2 * np.pi * (F * g["w"][:, None]).T @ F
            assert np.max(np.abs(G - np.eye(len(ls)))) < 1e-12, (m, sign)


def _draw(L, seed, nmaps=1):
    rng = np.random.default_rng(seed)
    n = _nalm(L, L)
    e = (rng.standard_normal((nmaps, n)) + 1j * rng.standard_normal((nmaps, n))) / np.sqrt(2)
    b = (rng.standard_normal((nmaps, n)) + 1j * rng.standard_normal((nmaps, n))) / np.sqrt(2)
    for l in range(L + 1):  # E_l0, B_l0 real (Q and U are real fields)
        e[:, _idx(l, 0, L)] = e[:, _idx(l, 0, L)].real
        b[:, _idx(l, 0, L)] = b[:, _idx(l, 0, L)].real
    for x in (e, b):        # no spin-2 content below l = 2
        for l in (0, 1):
            for m in range(0, min(l, L) + 1):
                x[:, _idx(l, m, L)] = 0
    return e, b


def test_spin2_synthesis_brute_force(oracle_mod, closed_forms):
    L = 4
    g = oracle_mod.healpix_grid(2)
    e, b = _draw(L, 71)
    q, u = oracle_mod.alm2map_spin2(g, L, L, e, b)
    th = np.repeat(np.arccos(g["x"]), g["nphi"])
    phi = np.concatenate([g["phi0"][r] + 2 * np.pi * np.arange(g["nphi"][r]) / g["nphi"][r]
                          for r in range(g["nrings"])])
    P = np.zeros(g["npix"], dtype=complex)
    for (l, m), (fp, _) in closed_forms.items():
        am = abs(m)
        if m >= 0:
            E, B = e[0, _idx(l, am, L)], b[0, _idx(l, am, L)]
        else:
            E, B = (-1) ** am * np.conj(e[0, _idx(l, am, L)]), (-1) ** am * np.conj(b[0, _idx(l, am, L)])
        P -= (E + 1j * B) * np.array([complex(fp(t)) for t in th]) * np.exp(1j * m * phi)
    assert np.max(np.abs(q[0] - P.real)) < 1e-12 * np.max(np.abs(P))
    assert np.max(np.abs(u[0] - P.imag)) < 1e-12 * np.max(np.abs(P))


def test_spin2_gauss_legendre_round_trip(oracle_mod):
    L = 24
    n, nphi = L + 2, 2 * L + 3
    g = oracle_mod.gl_grid(n, nphi)
    e, b = _draw(L, 72)
    q, u = oracle_mod.alm2map_spin2(g, L, L, e, b)
    P = (q[0] + 1j * u[0]).reshape(n, nphi)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    tabs = [oracle_mod.lam_spin2(L, L, g["x"][r], g["st"][r])[0] for r in range(n)]
    for m in range(0, L + 1):
        # -(E + iB)_lm = sum_r w_r (2 pi / nphi) sum_j P_rj 2lambda_lm(x_r) e^{-i m phi_j}
        pm = (P * np.exp(-1j * m * phi)[None, :]).sum(axis=1) * (2 * np.pi / nphi)
        for l in range(max(2, m), L + 1):
            c = -np.sum(g["w"] * pm * np.array([t[_idx(l, m, L)] for t in tabs]))
            want = e[0, _idx(l, m, L)] + 1j * b[0, _idx(l, m, L)]
            assert abs(c - want) < 1e-11, (l, m, c, want)


# ---- planted mistakes: each mutation of the oracle's spin-2 formula fails a pin

MUTATIONS = {
    "sign of the 2 m c term": ("(2.0 * mm * mm + 2.0 * mm * x)", "(2.0 * mm * mm - 2.0 * mm * x)"),
    "derivative recurrence coefficient": ("(2.0 * l + 1.0) * ((double)l * l - (double)m * m) / (2.0 * l - 1.0)",
                                          "(2.0 * l + 1.0) * ((double)l * l - (double)m * m) / (2.0 * l + 1.0)"),
    "normalisation K_l": ("(l - 1.0) * l * (l + 1.0) * (l + 2.0)", "(l - 1.0) * l * (l + 1.0) * (l + 1.0)"),
    "parity of negative orders": ("(sg && (m & 1)) ? -1.0 : 1.0", "1.0"),
    "sign of the first raising": ("-2.0 * (x + mm) * sDm * u", "-2.0 * (x - mm) * sDm * u"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_spin2_mistakes_fail_a_pin(oracle_mod, closed_forms, tmp_path, name):
    import ctypes
    import os
    import subprocess
    src = open(os.path.join(os.path.dirname(oracle_mod.__file__), "sht_oracle.c")).read()
    a, b = MUTATIONS[name]
    assert src.count(a) == 1, name
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(a, b))
    so = tmp_path / "mut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off", "-o", str(so),
                    str(mut), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    lib.orc_lambda_spin2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_void_p]
    L = 4
    caught = False
    for theta in (0.31, 0.9, 2.2):
        plus, minus = np.zeros(_nalm(L, L)), np.zeros(_nalm(L, L))
        lib.orc_lambda_spin2(L, L, math.cos(theta), math.sin(theta), plus.ctypes.data, minus.ctypes.data)
        for (l, m), (fp, _) in closed_forms.items():
            got = plus[_idx(l, abs(m), L)] if m >= 0 else minus[_idx(l, abs(m), L)]
            if abs(got - complex(fp(theta)).real) > 1e-9:
                caught = True
    assert caught, name
