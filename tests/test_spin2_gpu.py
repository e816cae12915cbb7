"""Spin-2 (Q/U polarisation) synthesis on the GPU, FP64, against the oracle's
literal sum over both signs of m (the GPU instead contracts the half sum and
half difference of the spin +-2 functions with E and B and runs the ring step
twice).  Normwise max error per map and component."""
import numpy as np
import pytest
import torch

from paper_1010_1260_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import sht as s
    s.lib()
    return s


def _nerr(got, want):
    ok = np.isfinite(want)
    return float(np.max(np.abs(got[ok] - want[ok])) / np.max(np.abs(want[ok])))


def _eb(lmax, mmax, seed, nmaps):
    e = inputs.batch_alm(lmax, mmax, seed, nmaps, "white")
    b = inputs.batch_alm(lmax, mmax, seed + 1000, nmaps, "white")
    return e, b


CASES = [
    ("hp", 8, 20, 20, 2),
    ("hp", 16, 40, 33, 3),
    ("gl", (32, 65), 31, 31, 2),
    ("rings", None, 24, 24, 2),
    ("hp", 64, 160, 160, 1),     # rings with aliasing (n_phi < 2 lmax + 1)
]


def _grid(oracle_mod, sht, kind, size):
    if kind == "hp":
        return oracle_mod.healpix_grid(size), sht.healpix(size)
    if kind == "gl":
        return oracle_mod.gl_grid(*size), sht.gl(*size)
    theta = np.array([0.2, 0.7, 1.2, 1.9, 2.6])
    nphi = np.array([9, 30, 48, 51, 12], dtype=np.int32)
    phi0 = np.array([0.1, 0.0, 0.5, 2.0, 0.3])
    return oracle_mod.rings_grid(theta, nphi, phi0), sht.rings(theta, nphi, phi0)


@pytest.mark.parametrize("case", CASES)
def test_spin2_matches_oracle(oracle_mod, sht, case):
    kind, size, lmax, mmax, nmaps = case
    og, sg = _grid(oracle_mod, sht, kind, size)
    e, b = _eb(lmax, mmax, 50 + lmax, nmaps)
    plan = sht.Plan(sg, lmax, mmax)
    got = plan.alm2map_spin2(torch.from_numpy(e).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    q, u = oracle_mod.alm2map_spin2(og, lmax, mmax, e, b)
    for k in range(nmaps):
        assert _nerr(got[k, 0], q[k]) < 1e-10
        assert _nerr(got[k, 1], u[k]) < 1e-10


def test_spin2_full_size_sampled_rings(oracle_mod, sht):
    """nside 1024, lmax 2048, 2 maps, on a stratified ring sample (poles, equator,
    belt and both kinds of cap ring)."""
    og, sg = oracle_mod.healpix_grid(1024), sht.healpix(1024)
    e = inputs.batch_alm(2048, 2048, 61, 2)
    b = inputs.batch_alm(2048, 2048, 62, 2)
    plan = sht.Plan(sg, 2048)
    got = plan.alm2map_spin2(torch.from_numpy(e).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    rings, _ = inputs.healpix_ring_sample(1024, 16, 5, n_large=4, n_smooth_cap=4)
    q, u = oracle_mod.alm2map_spin2(og, 2048, 2048, e, b, rings=rings)
    for k in range(2):
        assert _nerr(got[k, 0], q[k]) < 1e-9
        assert _nerr(got[k, 1], u[k]) < 1e-9


def test_spin2_batch_equals_singles(sht):
    plan = sht.Plan(sht.healpix(16), 30)
    e, b = _eb(30, 30, 7, 3)
    E, Bt = torch.from_numpy(e).cuda(), torch.from_numpy(b).cuda()
    batch = plan.alm2map_spin2(E, Bt)
    for k in range(3):
        assert torch.equal(plan.alm2map_spin2(E[k], Bt[k]), batch[k])


def test_spin2_pure_e_and_pure_b(sht):
    """Rotating E into B (B' = E, E' = -B) turns (Q, U) into (U, -Q)... as the
    definition's (E + iB) -> i (E + iB) multiplies Q + iU by i."""
    plan = sht.Plan(sht.healpix(16), 30)
    e, b = _eb(30, 30, 8, 1)
    E, Bt = torch.from_numpy(e).cuda(), torch.from_numpy(b).cuda()
    m1 = plan.alm2map_spin2(E, Bt)
    m2 = plan.alm2map_spin2(-Bt, E)
    scale = float(m1.abs().max())
    assert float((m2[0, 0] + m1[0, 1]).abs().max()) < 1e-12 * scale
    assert float((m2[0, 1] - m1[0, 0]).abs().max()) < 1e-12 * scale


def test_spin2_rejects_other_forms_and_polar_rings(sht):
    plan = sht.Plan(sht.healpix(4), 8)
    e = torch.zeros((1, plan.nalm), dtype=torch.complex128, device="cuda")
    out = torch.zeros((1, 2, plan.npix), dtype=torch.float64, device="cuda")
    L = sht.lib()
    assert L.sht_alm2map_spin2(plan.handle, 1, e.data_ptr(), e.data_ptr(), out.data_ptr(), sht.PREC["bf16x6_tc"],
                               None) == sht.SHT_EUNSUPPORTED
    polar = sht.Plan(sht.rings([0.0, 1.0], [4, 8], [0.0, 0.0]), 4)
    e4 = torch.zeros((1, polar.nalm), dtype=torch.complex128, device="cuda")
    with pytest.raises(sht.ShtError):
        polar.alm2map_spin2(e4, e4)
