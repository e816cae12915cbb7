"""map2alm_adjoint (the real-linear transpose of alm2map) on the GPU: against
the oracle's literal transpose, the dot-product identity, PyTorch autograd,
and central finite differences of a weighted least-squares loss."""
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


def _grids(oracle_mod, sht, kind, size):
    if kind == "hp":
        return oracle_mod.healpix_grid(size), sht.healpix(size)
    if kind == "gl":
        return oracle_mod.gl_grid(*size), sht.gl(*size)
    theta, nphi, phi0 = size
    return oracle_mod.rings_grid(theta, nphi, phi0), sht.rings(theta, nphi, phi0)


def _nerr(got, want):
    ok = np.isfinite(want)
    return np.max(np.abs(got[ok] - want[ok])) / np.max(np.abs(want[ok]))


def _dot(a, g, ms):
    a = np.where(ms == 0, a.real + 0j, a)
    return np.sum(a.real * g.real + a.imag * g.imag)


CASES = [
    ("hp", 1, 8, 8, 1),
    ("hp", 4, 8, 5, 2),
    ("hp", 16, 40, 40, 3),
    ("hp", 37, 70, 61, 5),
    ("gl", (9, 15), 7, 3, 2),
    ("gl", (300, 601), 299, 299, 1),   # > 128 pairs (three pair tiles), lmax + 1 not a multiple of 32
    ("hp", 6, 30, 0, 2),
    ("hp", 3, 0, 0, 1),
]


@pytest.mark.parametrize("case", CASES)
def test_adjoint_matches_oracle(oracle_mod, sht, case):
    kind, size, lmax, mmax, nmaps = case
    og, sg = _grids(oracle_mod, sht, kind, size)
    y = inputs.gaussian_map(og["npix"], 200 + lmax, nmaps)
    plan = sht.Plan(sg, lmax, mmax)
    got = plan.map2alm_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    want = oracle_mod.map2alm_adjoint(og, lmax, mmax, y)
    for b in range(nmaps):
        assert _nerr(got[b].view(np.float64), want[b].view(np.float64)) < 1e-10


def test_adjoint_gl_lmax127_oracle(oracle_mod, sht):
    """Oracle adjoint on the Gauss-Legendre 128 x 256 grid at lmax 127."""
    og, sg = _grids(oracle_mod, sht, "gl", (128, 256))
    y = inputs.gaussian_map(og["npix"], 5)
    got = sht.Plan(sg, 127).map2alm_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    want = oracle_mod.map2alm_adjoint(og, 127, 127, y)
    assert _nerr(got.view(np.float64), want.view(np.float64)) < 1e-10


def test_adjoint_generic_rings(oracle_mod, sht):
    theta = np.array([0.0, 0.05, 0.8, 1.3, np.pi / 2, 2.2, 3.0, np.pi])
    nphi = np.array([1, 5, 9, 12, 7, 30, 3, 2])
    phi0 = np.array([0.0, 0.3, -0.2, 0.0, 1.7, 0.05, 2.0, 0.4])
    og, sg = _grids(oracle_mod, sht, "rings", (theta, nphi, phi0))
    y = inputs.gaussian_map(og["npix"], 6, 2)
    got = sht.Plan(sg, 12, 10).map2alm_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    want = oracle_mod.map2alm_adjoint(og, 12, 10, y)
    assert _nerr(got.view(np.float64), want.view(np.float64)) < 1e-10


def test_adjoint_lmax2048_sampled_m(oracle_mod, sht):
    og, sg = _grids(oracle_mod, sht, "hp", 1024)
    y = inputs.gaussian_map(og["npix"], 7)
    got = sht.Plan(sg, 2048).map2alm_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()[0]
    ms_sel = [0, 1, 2, 511, 1024, 2047, 2048]
    want = oracle_mod.map2alm_adjoint(og, 2048, 2048, y, ms=ms_sel)[0]
    _, ms = inputs.lm_arrays(2048, 2048)
    sel = np.isin(ms, ms_sel)
    assert _nerr(got[sel].view(np.float64), want[sel].view(np.float64)) < 1e-10


@pytest.mark.parametrize("nside,lmax,nmaps", [(4, 9, 1), (64, 130, 3), (1024, 2048, 2)])
def test_dot_product_identity(sht, nside, lmax, nmaps):
    plan = sht.Plan(sht.healpix(nside), lmax)
    a = torch.from_numpy(inputs.batch_alm(lmax, lmax, 8, nmaps, spectrum="white")).cuda()
    y = torch.from_numpy(inputs.gaussian_map(plan.npix, 9, nmaps)).cuda()
    ya = plan.alm2map(a)
    g = plan.map2alm_adjoint(y)
    _, ms = inputs.lm_arrays(lmax, lmax)
    for b in range(nmaps):
        lhs = float(torch.dot(ya[b], y[b]))
        rhs = _dot(a[b].cpu().numpy(), g[b].cpu().numpy(), ms)
        scale = float(torch.linalg.norm(ya[b]) * torch.linalg.norm(y[b]))
        assert abs(lhs - rhs) < 1e-12 * scale


def test_adjoint_batch_equals_singles(sht):
    plan = sht.Plan(sht.healpix(16), 47)
    y = torch.from_numpy(inputs.gaussian_map(plan.npix, 10, 6)).cuda()
    batch = plan.map2alm_adjoint(y)
    for b in range(6):
        assert torch.equal(plan.map2alm_adjoint(y[b]), batch[b])


def test_autograd_gradcheck_tiny(sht):
    from paper_1010_1260_gb300.autograd import alm2map
    plan = sht.Plan(sht.healpix(2), 4)
    a = torch.from_numpy(inputs.gaussian_alm(4, 4, 11, spectrum="white")).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: alm2map(t, plan), (a,), eps=1e-6, atol=1e-8)


def _loss(plan, a, w, d):
    from paper_1010_1260_gb300.autograd import alm2map
    s = alm2map(a, plan)
    return torch.sum(w * (s - d) ** 2)


@pytest.mark.parametrize("nside,lmax,nmaps", [(64, 128, 2), (1024, 2048, 16)])
def test_finite_differences_weighted_loss(sht, nside, lmax, nmaps):
    """loss = sum_p w_p (alm2map(a)_p - d_p)^2, w ~ U(0.5, 1.5), d ~ N(0, 1):
    autograd gradient vs central differences on 32 random coefficients.  The
    loss is quadratic in a, so central differences carry no truncation error
    and the step can be large (only rounding in the loss sum remains)."""
    plan = sht.Plan(sht.healpix(nside), lmax)
    a0 = torch.from_numpy(inputs.batch_alm(lmax, lmax, 5, nmaps)).cuda()
    w_np, d_np = inputs.loss_weights(plan.npix, 5, nmaps)
    w = torch.from_numpy(w_np).cuda()
    d = torch.from_numpy(d_np).cuda()
    a = a0.clone().requires_grad_(True)
    L = _loss(plan, a, w, d)
    L.backward()
    grad = a.grad.detach()
    rng = np.random.default_rng(6)
    h = 1e-2
    worst = 0.0
    for _ in range(32):
        b = int(rng.integers(nmaps))
        i = int(rng.integers(plan.nalm))
        comp = int(rng.integers(2))
        if i <= lmax and comp == 1:
            comp = 0                     # Im of m = 0 does not enter the map
        e = torch.zeros_like(a0)
        e[b, i] = h if comp == 0 else 1j * h
        with torch.no_grad():
            lp = float(_loss(plan, a0 + e, w, d))
            lm = float(_loss(plan, a0 - e, w, d))
        fd = (lp - lm) / (2 * h)
        an = float(grad[b, i].real if comp == 0 else grad[b, i].imag)
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-3 * float(L.detach()) / plan.npix))
    assert worst < 1e-6, worst
