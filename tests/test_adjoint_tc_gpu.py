"""Tensor-core transpose (map2alm_adjoint in the BF16 forms) on the GPU: the
Legendre step reads the plan-time Lambda operand transposed (MN-major) and
contracts over the ring pairs on the tensor cores, after an FP32 ring
analysis.  Checked against the oracle's literal transpose map by map, the
dot-product identity with the forward of the same form, the full-size
workload on sampled orders, and the autograd routing."""
import numpy as np
import pytest
import torch

from paper_1010_1260_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"bf16x6_tc": 1e-6, "bf16x3_tc": 3e-5}   # relative L2 per map, as the forward forms


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import sht as s
    s.lib()
    return s


def _grids(oracle_mod, sht, kind, size):
    if kind == "hp":
        return oracle_mod.healpix_grid(size), sht.healpix(size)
    return oracle_mod.gl_grid(*size), sht.gl(*size)


def _rl2(got, want):
    g, w = got.view(np.float64), want.view(np.float64)
    return float(np.linalg.norm(g - w) / np.linalg.norm(w))


CASES = [
    ("hp", 16, 40, 40, 3),
    ("hp", 37, 70, 61, 5),
    ("hp", 6, 30, 0, 2),                # mmax 0
    ("gl", (300, 601), 299, 299, 2),    # 150 pairs: a partial ring block and chunk
    ("hp", 64, 160, 160, 20),           # 20 maps: 64 operand columns
    ("hp", 32, 80, 80, 33),             # 33 maps: two launches of the contraction
]


@pytest.mark.parametrize("prec", ["bf16x6_tc", "bf16x3_tc"])
@pytest.mark.parametrize("case", CASES)
def test_adjoint_tc_matches_oracle(oracle_mod, sht, case, prec):
    kind, size, lmax, mmax, nmaps = case
    og, sg = _grids(oracle_mod, sht, kind, size)
    y = inputs.gaussian_map(og["npix"], 300 + lmax, nmaps).astype(np.float32)
    plan = sht.Plan(sg, lmax, mmax)
    plan.lambda_cache(prec)
    got = plan.map2alm_adjoint(torch.from_numpy(y).cuda(), prec).cpu().numpy()
    want = oracle_mod.map2alm_adjoint(og, lmax, mmax, y.astype(np.float64))
    for b in range(nmaps):
        assert _rl2(got[b], want[b]) < TOL[prec], (b, _rl2(got[b], want[b]))
    _, ms = inputs.lm_arrays(lmax, mmax)
    assert np.all(got[:, ms == 0].imag == 0)


def test_adjoint_tc_generic_rings(oracle_mod, sht):
    """Rings at arbitrary colatitudes with arbitrary phi0 (phases by sincos),
    odd and even lengths, a ring on each pole, and ring weights for map2alm."""
    theta = np.array([0.0, 0.05, 0.3, 0.8, 1.3, np.pi / 2, 1.9, 2.2, 2.9, np.pi])
    nphi = np.array([1, 7, 24, 33, 50, 61, 48, 40, 11, 2])
    phi0 = np.array([0.0, 0.3, -0.2, 0.0, 1.7, 0.05, 2.0, 0.4, 0.9, 0.1])
    og = oracle_mod.rings_grid(theta, nphi, phi0)
    plan = sht.Plan(sht.rings(theta, nphi, phi0), 24, 20)
    plan.lambda_cache("bf16x6_tc")
    y = inputs.gaussian_map(og["npix"], 15, 3).astype(np.float32)
    got = plan.map2alm_adjoint(torch.from_numpy(y).cuda(), "bf16x6_tc").cpu().numpy()
    want = oracle_mod.map2alm_adjoint(og, 24, 20, y.astype(np.float64))
    for b in range(3):
        assert _rl2(got[b], want[b]) < 1e-6
    w = np.linspace(0.5, 1.5, len(theta))
    plan.set_ring_weights(w)
    got = plan.map2alm(torch.from_numpy(y).cuda(), prec="bf16x6_tc").cpu().numpy()
    want = oracle_mod.map2alm(og, 24, 20, y.astype(np.float64), weights=w)
    for b in range(3):
        assert _rl2(got[b], want[b]) < 1e-6


def test_adjoint_tc_skip_off_same(sht):
    """The chunks the skip leaves out hold only zeros: same result without it."""
    plan = sht.Plan(sht.healpix(64), 160)
    plan.lambda_cache("bf16x6_tc")
    y = torch.from_numpy(inputs.gaussian_map(plan.npix, 11, 4).astype(np.float32)).cuda()
    g1 = plan.map2alm_adjoint(y, "bf16x6_tc")
    plan.skip_evanescent(False)
    g2 = plan.map2alm_adjoint(y, "bf16x6_tc")
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)


@pytest.mark.parametrize("nside,lmax,nmaps", [(16, 40, 2), (64, 130, 3)])
def test_adjoint_tc_dot_product(sht, nside, lmax, nmaps):
    prec = "bf16x6_tc"
    plan = sht.Plan(sht.healpix(nside), lmax)
    plan.lambda_cache(prec)
    a = torch.from_numpy(inputs.batch_alm(lmax, lmax, 8, nmaps, spectrum="white")).cuda()
    y = torch.from_numpy(inputs.gaussian_map(plan.npix, 9, nmaps).astype(np.float32)).cuda()
    ya = plan.alm2map(a, prec).double()
    g = plan.map2alm_adjoint(y, prec).cpu().numpy()
    _, ms = inputs.lm_arrays(lmax, lmax)
    for b in range(nmaps):
        lhs = float(torch.dot(ya[b], y[b].double()))
        ab = a[b].cpu().numpy()
        ab = np.where(ms == 0, ab.real + 0j, ab)
        rhs = float(np.sum(ab.real * g[b].real + ab.imag * g[b].imag))
        scale = float(torch.linalg.norm(ya[b]) * torch.linalg.norm(y[b].double()))
        assert abs(lhs - rhs) < 2e-6 * scale


def test_adjoint_tc_full_size_sampled_m(oracle_mod, sht):
    """HEALPix nside 1024, lmax 2048, 16 maps (the differentiation workload)."""
    og, sg = _grids(oracle_mod, sht, "hp", 1024)
    plan = sht.Plan(sg, 2048)
    plan.lambda_cache("bf16x6_tc")
    y = inputs.gaussian_map(og["npix"], 7, 16).astype(np.float32)
    got = plan.map2alm_adjoint(torch.from_numpy(y).cuda(), "bf16x6_tc").cpu().numpy()
    ms_sel = [0, 1, 2, 511, 1024, 2047, 2048]
    _, ms = inputs.lm_arrays(2048, 2048)
    sel = np.isin(ms, ms_sel)
    for b in (0, 15):
        want = oracle_mod.map2alm_adjoint(og, 2048, 2048, y[b:b + 1].astype(np.float64), ms=ms_sel)[0]
        assert _rl2(got[b][sel], want[sel]) < 1e-6


def test_adjoint_tc_needs_operand_and_bf16(sht):
    plan = sht.Plan(sht.healpix(16), 40)
    y = torch.from_numpy(inputs.gaussian_map(plan.npix, 3).astype(np.float32)).cuda()
    with pytest.raises(Exception, match="sht_lambda_cache"):
        plan.map2alm_adjoint(y, "bf16x6_tc")
    plan.lambda_cache("fp32_tc")
    with pytest.raises(Exception, match="BF16"):
        plan.map2alm_adjoint(y, "fp32_tc")


def test_autograd_routes_to_tc_adjoint(sht):
    from paper_1010_1260_gb300 import autograd
    plan = sht.Plan(sht.healpix(32), 64)
    a = torch.from_numpy(inputs.batch_alm(64, 64, 12, 2)).cuda().requires_grad_(True)
    w = torch.from_numpy(inputs.gaussian_map(plan.npix, 13, 2).astype(np.float32)).cuda()
    plan.lambda_cache("bf16x6_tc")
    s = autograd.alm2map(a, plan, "bf16x6_tc")
    (s * w).sum().backward()
    want = plan.map2alm_adjoint(w, "bf16x6_tc")
    torch.cuda.synchronize()
    assert torch.equal(a.grad, want)


def test_map2alm_tc_matches_oracle(oracle_mod, sht):
    """Quadrature-weighted analysis in the BF16x6 form (one pass): the exact
    inverse on a Gauss-Legendre grid, and the oracle on HEALPix."""
    prec = "bf16x6_tc"
    og, sg = _grids(oracle_mod, sht, "gl", (64, 129))
    plan = sht.Plan(sg, 63)
    plan.lambda_cache(prec)
    a = inputs.batch_alm(63, 63, 21, 3)
    y = plan.alm2map(torch.from_numpy(a).cuda(), prec)       # float32 maps
    got = plan.map2alm(y, prec=prec).cpu().numpy()
    for b in range(3):
        assert _rl2(got[b], a[b]) < 2e-6
    og, sg = _grids(oracle_mod, sht, "hp", 32)
    plan = sht.Plan(sg, 64)
    plan.lambda_cache(prec)
    y = inputs.gaussian_map(og["npix"], 22, 2).astype(np.float32)
    got = plan.map2alm(torch.from_numpy(y).cuda(), prec=prec).cpu().numpy()
    want = oracle_mod.map2alm(og, 64, 64, y.astype(np.float64))
    for b in range(2):
        assert _rl2(got[b], want[b]) < 1e-6
    with pytest.raises(Exception, match="niter"):
        plan.map2alm(torch.from_numpy(y).cuda(), niter=1, prec=prec)


def test_adjoint_tc_analysis_tiles_bit_identical(sht):
    """The FP32 ring analysis gives the same bits for every maps-per-CTA tile."""
    plan = sht.Plan(sht.healpix(32), 64)
    plan.lambda_cache("bf16x6_tc")
    y = torch.from_numpy(inputs.gaussian_map(plan.npix, 14, 11).astype(np.float32)).cuda()
    assert plan.tiles()["fp32_analysis_maps"] == 8
    ref = plan.map2alm_adjoint(y, "bf16x6_tc")
    for g in (1, 2, 4):
        plan.set_tiles(fp32_analysis_maps=g)
        got = plan.map2alm_adjoint(y, "bf16x6_tc")
        torch.cuda.synchronize()
        assert torch.equal(got, ref), g
    with pytest.raises(sht.ShtError):
        plan.set_tiles(fp32_analysis_maps=3)


def test_finite_differences_tc_backward(sht):
    """The weighted least-squares loss through autograd with the BF16x6 forward
    (from the Lambda operand) and the tensor-core transpose as backward,
    against central differences of the same loss on 16 random coefficients.
    The loss is quadratic in a, so central differences carry no truncation
    error and a unit step only meets the FP32 rounding of the maps."""
    from paper_1010_1260_gb300 import autograd
    nside, lmax, nmaps = 64, 128, 2
    plan = sht.Plan(sht.healpix(nside), lmax)
    plan.lambda_cache("bf16x6_tc")
    a0 = torch.from_numpy(inputs.batch_alm(lmax, lmax, 5, nmaps)).cuda()
    w_np, d_np = inputs.loss_weights(plan.npix, 5, nmaps)
    w = torch.from_numpy(w_np).cuda()
    d = torch.from_numpy(d_np).cuda()

    def loss(a):
        s = autograd.alm2map(a, plan, "bf16x6_tc")
        return (w * (s.double() - d) ** 2).sum()

    a = a0.clone().requires_grad_(True)
    L = loss(a)
    L.backward()
    grad = a.grad.detach()
    rng = np.random.default_rng(16)
    h = 1.0
    worst = 0.0
    for _ in range(16):
        b = int(rng.integers(nmaps))
        i = int(rng.integers(plan.nalm))
        comp = int(rng.integers(2))
        if i <= lmax and comp == 1:
            comp = 0
        e = torch.zeros_like(a0)
        e[b, i] = h if comp == 0 else 1j * h
        with torch.no_grad():
            fd = (float(loss(a0 + e)) - float(loss(a0 - e))) / (2 * h)
        an = float(grad[b, i].real if comp == 0 else grad[b, i].imag)
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-3 * float(L.detach()) / plan.npix))
    assert worst < 1e-4, worst
