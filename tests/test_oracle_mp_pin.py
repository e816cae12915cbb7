"""Extended-precision pin of the oracle's exponent-tracked recurrence.

lambda_lm(cos theta) is recomputed with mpmath at 40 significant digits by the
textbook normalised three-term recurrence (mpmath numbers have no underflow,
so no rescaling is needed), for every degree up to lmax = 2048 at several
orders and colatitudes -- including the deep evanescent region near the
pole, where lambda_mm is far below the FP64 range and the oracle only reaches
the representable values through its power-of-two exponent tracking
(Algorithm 2).  The oracle must agree wherever the value is an FP64 normal
number, and give zero (or a subnormal) where it is not.  The small-degree
values are also checked against mpmath's own associated Legendre function
(its hypergeometric evaluation, a different method)."""
import math

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")


def _idx(l, m, L):
    return m * (2 * L + 3 - m) // 2 + (l - m)


def _lam_mp(L, m, x, s):
    """[lambda_lm for l = m..L] as mpf for the given FP64 inputs x = cos theta
    and s = sin theta taken exactly (so that only the arithmetic differs from
    the oracle's, not the rounding of the inputs), Condon-Shortley phase
    included."""
    mp = mpmath.mp
    x = mpmath.mpf(x)
    s = mpmath.mpf(s)
    v = mpmath.sqrt(1 / (4 * mp.pi))
    for k in range(1, m + 1):
        v *= -mpmath.sqrt(mpmath.mpf(2 * k + 1) / (2 * k)) * s
    out = [v]
    if m + 1 <= L:
        out.append(x * mpmath.sqrt(2 * m + 3) * v)
    for l in range(m + 2, L + 1):
        a = mpmath.sqrt(mpmath.mpf(4 * l * l - 1) / (l * l - m * m))
        b = mpmath.sqrt(mpmath.mpf((l - 1) ** 2 - m * m) / (4 * (l - 1) ** 2 - 1))
        out.append(a * (x * out[-1] - b * out[-2]))
    return out


def test_small_degrees_against_mpmath_legenp(oracle_mod):
    mpmath.mp.dps = 30
    L = 12
    for theta in (0.2, 1.1, 2.6):
        lam = oracle_mod.lam(L, L, math.cos(theta), math.sin(theta))
        for m in range(0, L + 1):
            for l in range(m, L + 1):
                p = mpmath.legenp(l, m, mpmath.cos(theta), type=2)
                ref = mpmath.sqrt((2 * l + 1) / (4 * mpmath.pi) * mpmath.factorial(l - m) /
                                  mpmath.factorial(l + m)) * p
                assert abs(lam[_idx(l, m, L)] - float(ref)) < 1e-13 * max(1.0, abs(float(ref))), (l, m, theta)


@pytest.mark.parametrize("theta", [0.002, 0.02, 0.3, 1.2, math.pi / 2])
def test_recurrence_against_extended_precision_lmax_2048(oracle_mod, theta):
    mpmath.mp.dps = 40
    L = 2048
    x, st = math.cos(theta), math.sin(theta)
    lam = oracle_mod.lam(L, L, x, st)
    tiny = 2.0 ** -1022
    worst = 0.0
    checked = 0
    for m in (0, 1, 37, 500, 1000, 1500, 2047, 2048):
        ref = _lam_mp(L, m, x, st)
        mag = np.array([float(abs(v)) for v in ref])
        for l in range(m, L + 1):
            got = lam[_idx(l, m, L)]
            r = ref[l - m]
            # error relative to the local envelope: the recurrence oscillates
            # past the turning point, where single values pass through zero
            env = mag[max(0, l - m - 16): l - m + 17].max()
            if abs(r) >= tiny * 2 ** 60:
                rel = abs(got - float(r)) / env
                worst = max(worst, rel)
                checked += 1
            elif abs(r) < tiny:
                assert abs(got) < tiny, (l, m, got, r)
    assert checked > 0
    # FP64 rounding of the forward recurrence grows with the degree; it is worst
    # next to the pole at small m (measured 6e-11 at theta = 0.002, m = 1,
    # l = 1915; elsewhere below 4e-12), far below what a wrong coefficient,
    # sign or rescaling would give (errors of order 1/l or 2^400)
    assert worst < (1e-9 if theta < 0.01 else 2e-11), worst


MUTATIONS = {
    "l_{l-2} not rescaled with l_{l-1}": ("l0 = ldexp(l0, -ORC_S);\n                    k += 1;",
                                         "k += 1;"),
    "exponent stepped the wrong way": ("l0 = ldexp(l0, -ORC_S);\n                    k += 1;",
                                       "l0 = ldexp(l0, -ORC_S);\n                    k -= 1;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_tracking_mistakes_fail_the_pin(oracle_mod, tmp_path, name):
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
    lib.orc_lambda.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               ctypes.c_void_p]
    mpmath.mp.dps = 40
    L, theta, m = 2048, 0.3, 500
    x, st = math.cos(theta), math.sin(theta)
    out = np.zeros((L + 1) * (L + 2) // 2)
    lib.orc_lambda(L, L, x, st, 1, out.ctypes.data)
    ref = _lam_mp(L, m, x, st)
    bad = 0
    for l in range(m, L + 1):
        r = float(ref[l - m])
        if abs(r) > 1e-250 and abs(out[_idx(l, m, L)] - r) > 1e-6 * abs(r):
            bad += 1
    assert bad > 0, name
