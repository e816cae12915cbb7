"""Precision forms of alm2map on the GPU: FP64 recurrence, tensor-core
contraction (3xTF32, split-BF16 with 3 products, BF16 with 3 pieces and 6
products), FP32 ring step.  Error per map is the relative L2 norm against the
FP64 oracle, ||s - s_ref||_2 / ||s_ref||_2; targets: 1e-5 for the TF32 form,
1e-6 for the BF16 forms.  The 3-product BF16 form (two 8-bit pieces, about 16
significant bits) does NOT meet the 1e-6 target (it measures about 4.9e-6);
it is checked against the bound its pieces allow, 3e-5, and the 6-product
form is the one that meets 1e-6."""
import numpy as np
import pytest
import torch

from paper_1010_1260_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp32_tc": 1e-5, "bf16x3_tc": 3e-5, "bf16x6_tc": 1e-6}


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import sht as s
    s.lib()
    return s


def _rl2(got, want):
    ok = np.isfinite(want)
    return float(np.linalg.norm(got[ok] - want[ok]) / np.linalg.norm(want[ok]))


def _grids(oracle_mod, sht, kind, size):
    if kind == "hp":
        return oracle_mod.healpix_grid(size), sht.healpix(size)
    return oracle_mod.gl_grid(*size), sht.gl(*size)


CASES = [
    ("hp", 16, 40, 40, 3),
    ("hp", 37, 70, 61, 1),      # 74 ring pairs (< 128), lmax - m not a multiple of the stage
    ("hp", 8, 100, 100, 33),    # aliasing; 66 columns -> N = 96
    ("gl", (128, 256), 127, 127, 2),
    ("hp", 64, 130, 130, 65),   # two launch groups (64 + 1 maps), 255 rings -> 2 ring blocks
    ("hp", 128, 256, 256, 4),   # belt rings of 512 pixels: direct FFT of length 256
    ("gl", (64, 2048), 63, 63, 2),    # rings of 2048 pixels: direct FFT of length 1024
    ("gl", (16, 8192), 15, 15, 2),    # rings of 8192 pixels: direct FFT of length 4096, maps in two rounds
]


@pytest.mark.parametrize("prec", ["fp32_tc", "bf16x3_tc", "bf16x6_tc"])
@pytest.mark.parametrize("case", CASES)
def test_tc_forms_vs_oracle(oracle_mod, sht, case, prec):
    kind, size, lmax, mmax, nmaps = case
    og, sg = _grids(oracle_mod, sht, kind, size)
    alm = inputs.batch_alm(lmax, mmax, 300 + lmax, nmaps)
    plan = sht.Plan(sg, lmax, mmax)
    got = plan.alm2map(torch.from_numpy(alm).cuda(), prec)
    plan.sync()
    got = got.double().cpu().numpy()
    want = oracle_mod.alm2map(og, lmax, mmax, alm)
    errs = [_rl2(got[b], want[b]) for b in range(nmaps)]
    assert max(errs) < TOL[prec], (prec, max(errs))


@pytest.mark.parametrize("prec", ["fp32_tc", "bf16x6_tc"])
def test_tc_full_size_sampled_rings(oracle_mod, sht, prec):
    """HEALPix nside 1024, lmax 2048, a batch of 64 maps (the benchmark's
    workload): every map checked, per map, on a ring sample stratified by ring
    class -- both poles, the equator, belt rings, polar-cap rings whose length
    has a prime factor >= 29 and cap rings whose length has none."""
    og, sg = _grids(oracle_mod, sht, "hp", 1024)
    alm = inputs.batch_alm(2048, 2048, 3, 64)
    plan = sht.Plan(sg, 2048)
    out = plan.alm2map(torch.from_numpy(alm).cuda(), prec)
    plan.sync()
    rings, cls = inputs.healpix_ring_sample(1024, 32, 33, n_large=8, n_smooth_cap=6)
    assert sorted(set(cls.values())) == ["belt", "cap_large_prime", "cap_smooth", "equator", "pole"]
    want = oracle_mod.alm2map(og, 2048, 2048, alm, rings=rings)
    got = out.double().cpu().numpy()
    errs = [_rl2(got[b], want[b]) for b in range(64)]
    assert max(errs) < TOL[prec], (prec, max(errs))


def test_tc_batch_equals_singles(sht):
    plan = sht.Plan(sht.healpix(16), 47)
    alm = torch.from_numpy(inputs.batch_alm(47, 47, 9, 5)).cuda()
    batch = plan.alm2map(alm, "fp32_tc")
    for b in range(5):
        single = plan.alm2map(alm[b], "fp32_tc")
        assert torch.allclose(single, batch[b], rtol=0, atol=1e-6 * float(batch[b].abs().max()))
    plan.sync()


def _rings_case():
    # generic rings: odd and even lengths, a prime length 61 (Bluestein, N = 61),
    # 2 x 31 (Bluestein, N = 31), arbitrary first azimuths (no table phases)
    theta = np.array([0.21, 0.47, 0.8, 1.1, 1.4, 1.7, 2.05, 2.5, 2.9])
    nphi = np.array([7, 61, 62, 90, 125, 124, 64, 33, 12], dtype=np.int32)
    phi0 = np.array([0.013, 0.4, 1.7, 0.0, 2.2, 0.31, 0.05, 3.0, 0.77])
    return theta, nphi, phi0


@pytest.mark.parametrize("prec", ["fp32_tc", "bf16x6_tc"])
@pytest.mark.parametrize("gl_odd", [False, True])
def test_tc_odd_lengths_and_generic_rings(oracle_mod, sht, prec, gl_odd):
    if gl_odd:
        lmax, nmaps = 30, 3
        og, sg = oracle_mod.gl_grid(31, 61), sht.gl(31, 61)       # odd n: full-length complex DFT
    else:
        lmax, nmaps = 40, 5
        theta, nphi, phi0 = _rings_case()
        og, sg = oracle_mod.rings_grid(theta, nphi, phi0), sht.rings(theta, nphi, phi0)
    alm = inputs.batch_alm(lmax, lmax, 400 + lmax, nmaps)
    plan = sht.Plan(sg, lmax)
    got = plan.alm2map(torch.from_numpy(alm).cuda(), prec)
    plan.sync()
    want = oracle_mod.alm2map(og, lmax, lmax, alm)
    g = got.double().cpu().numpy()
    errs = [_rl2(g[b], want[b]) for b in range(nmaps)]
    assert max(errs) < TOL[prec], errs
    # every tile shape gives the same maps on these rings too
    for gs, gb, nt in ((1, 1, 256), (4, 2, 512)):
        plan.set_tiles(ring_maps_smooth=gs, ring_maps_bluestein=gb, ring_threads=nt)
        again = plan.alm2map(torch.from_numpy(alm).cuda(), prec)
        plan.sync()
        assert torch.equal(again, got)


def test_host_stream_matches_device_calls(sht):
    """The pipelined host-buffer API gives the maps of one alm2map per batch."""
    plan = sht.Plan(sht.healpix(16), 40)
    batches = [torch.from_numpy(inputs.batch_alm(40, 40, 600 + k, 3)).pin_memory() for k in range(5)]
    outs = plan.alm2map_host_stream(batches, "bf16x6_tc")
    for k, a in enumerate(batches):
        want = plan.alm2map(a.cuda(), "bf16x6_tc").cpu()
        assert torch.equal(outs[k], want)
    # output buffers reused two apart, as the benchmark does
    pins = [torch.empty((3, plan.npix), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    outs = plan.alm2map_host_stream(batches[:4], "bf16x6_tc", outs=[pins[k % 2] for k in range(4)])
    assert torch.equal(pins[1], plan.alm2map(batches[3].cuda(), "bf16x6_tc").cpu())
