"""alm2map on the GPU (FP64 path) against the CPU oracle, element by element.

Tolerance: the FP64 path must match the oracle to 1e-10 in normwise max
relative error, max_p |s - s_ref| / max_p |s_ref|, per map.
"""
import numpy as np
import pytest
import torch

from paper_1010_1260_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import sht as s
    s.lib()
    return s


def _err(got, want):
    got = np.atleast_2d(got)
    want = np.atleast_2d(want)
    out = []
    for g, w in zip(got, want):
        ok = np.isfinite(w)
        out.append(np.max(np.abs(g[ok] - w[ok])) / max(np.max(np.abs(w[ok])), 1e-300))
    return max(out)


def _grids(oracle_mod, sht, kind, size):
    if kind == "hp":
        return oracle_mod.healpix_grid(size), sht.healpix(size)
    if kind == "gl":
        return oracle_mod.gl_grid(*size), sht.gl(*size)
    theta, nphi, phi0 = size
    return oracle_mod.rings_grid(theta, nphi, phi0), sht.rings(theta, nphi, phi0)


CASES = [
    ("hp", 1, 8, 8, 1),
    ("hp", 2, 8, 8, 1),
    ("hp", 4, 8, 5, 3),
    ("hp", 16, 40, 40, 2),         # ragged: lmax + 1 not a multiple of the l-chunk
    ("hp", 8, 100, 100, 1),        # heavy aliasing: n_phi <= 32 << 2 lmax + 1
    ("hp", 37, 70, 61, 5),         # odd nside: prime cap lengths
    ("gl", (8, 16), 7, 7, 1),
    ("gl", (9, 15), 7, 3, 2),      # odd ring count (equator ring unpaired), odd n_phi
    ("gl", (130, 259), 129, 129, 9),  # > 128 ring pairs: two ring blocks; 9 maps: two map groups
    ("hp", 3, 0, 0, 1),            # lmax = 0
    ("hp", 6, 30, 0, 2),           # mmax = 0
    ("hp", 5, 1, 1, 1),
]


@pytest.mark.parametrize("case", CASES)
def test_alm2map_fp64_small(oracle_mod, sht, case):
    kind, size, lmax, mmax, nmaps = case
    og, sg = _grids(oracle_mod, sht, kind, size)
    alm = inputs.batch_alm(lmax, mmax, 100 + lmax, nmaps, spectrum="white")
    plan = sht.Plan(sg, lmax, mmax)
    assert plan.npix == og["npix"] and plan.nalm == alm.shape[1]
    got = plan.alm2map(torch.from_numpy(alm).cuda()).cpu().numpy()
    want = oracle_mod.alm2map(og, lmax, mmax, alm)
    assert _err(got, want) < TOL64


def test_alm2map_generic_rings(oracle_mod, sht):
    theta = np.array([0.0, 0.05, 0.8, 1.3, np.pi / 2, 2.2, 3.0, np.pi])
    nphi = np.array([1, 5, 9, 12, 7, 30, 3, 2])
    phi0 = np.array([0.0, 0.3, -0.2, 0.0, 1.7, 0.05, 2.0, 0.4])
    og, sg = _grids(oracle_mod, sht, "rings", (theta, nphi, phi0))
    alm = inputs.batch_alm(12, 10, 5, 2, spectrum="white")
    got = sht.Plan(sg, 12, 10).alm2map(torch.from_numpy(alm).cuda()).cpu().numpy()
    want = oracle_mod.alm2map(og, 12, 10, alm)
    assert _err(got, want) < TOL64


def test_gl_cfg1(oracle_mod, sht):
    """Gauss-Legendre 128 rings x 256 pixels, lmax = mmax = 127, one map."""
    og, sg = _grids(oracle_mod, sht, "gl", (128, 256))
    alm = inputs.gaussian_alm(127, 127, 1, spectrum="white")
    got = sht.Plan(sg, 127).alm2map(torch.from_numpy(alm).cuda()).cpu().numpy()
    want = oracle_mod.alm2map(og, 127, 127, alm)
    assert _err(got, want) < TOL64


def test_healpix_cfg2_full_map(oracle_mod, sht):
    """HEALPix nside 512 (2047 rings, 3,145,728 pixels), lmax = mmax = 1024, one map."""
    og, sg = _grids(oracle_mod, sht, "hp", 512)
    alm = inputs.gaussian_alm(1024, 1024, 2, spectrum="cl")
    got = sht.Plan(sg, 1024).alm2map(torch.from_numpy(alm).cuda()).cpu().numpy()
    want = oracle_mod.alm2map(og, 1024, 1024, alm)
    assert _err(got, want) < TOL64


def test_healpix_lmax2048_sampled_rings(oracle_mod, sht):
    """HEALPix nside 1024, lmax 2048 (the batched workload's size), 2 maps,
    checked on a seeded sample of rings that holds both poles and the equator."""
    og, sg = _grids(oracle_mod, sht, "hp", 1024)
    alm = inputs.batch_alm(2048, 2048, 3, 2)
    got = sht.Plan(sg, 2048).alm2map(torch.from_numpy(alm).cuda()).cpu().numpy()
    rings = inputs.sample_rings(og["nrings"], 12, 31)
    want = oracle_mod.alm2map(og, 2048, 2048, alm, rings=rings)
    assert _err(got, want) < TOL64


def test_batch_equals_singles_bitwise(sht):
    plan = sht.Plan(sht.healpix(16), 47)
    alm = torch.from_numpy(inputs.batch_alm(47, 47, 9, 11, spectrum="white")).cuda()
    batch = plan.alm2map(alm)
    for b in range(alm.shape[0]):
        single = plan.alm2map(alm[b])
        assert torch.equal(single, batch[b])


def test_empty_batch_is_noop(sht):
    plan = sht.Plan(sht.healpix(4), 8)
    alm = torch.zeros((0, plan.nalm), dtype=torch.complex128, device="cuda")
    out = plan.alm2map(alm)
    assert out.shape == (0, plan.npix)


def test_imag_of_m0_is_ignored(sht):
    plan = sht.Plan(sht.healpix(4), 8)
    alm = torch.from_numpy(inputs.gaussian_alm(8, 8, 3, spectrum="white")).cuda()
    a2 = alm.clone()
    a2[0, :9] += 1j * torch.arange(9, device="cuda", dtype=torch.float64)
    assert torch.equal(plan.alm2map(alm), plan.alm2map(a2))


def test_null_pointers_rejected(sht):
    plan = sht.Plan(sht.healpix(4), 8)
    rc = sht.lib().sht_alm2map_batch(plan.handle, 1, None, None, 0, None)
    assert rc == sht.SHT_EINVAL
