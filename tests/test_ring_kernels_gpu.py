"""The two FP32 ring-step kernels of the tensor-core forms (Eq. Delta2map):
the register-FFT kernel (power-of-two lengths directly, other lengths by
Bluestein's algorithm with a power-of-two length, Delta blocks brought in by
tensor-map copies) and the shared-memory mixed-radix kernel.  Every kernel
choice meets the form's tolerance against the FP64 oracle on ring lengths that
exercise each path: direct lengths 256, 1024 and 4096 (two rounds of one map),
Bluestein lengths from 256 to 4096, odd map counts (asynchronous-copy
staging) and heavy aliasing."""
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


def _rl2(got, want):
    ok = np.isfinite(want)
    return float(np.linalg.norm(got[ok] - want[ok]) / np.linalg.norm(want[ok]))


CASES = [
    ("hp", 128, 256, 256, 4),        # belt N = 256 (direct), caps Bluestein 256..512
    ("hp", 16, 40, 40, 3),           # odd map count: asynchronous-copy staging
    ("hp", 8, 100, 100, 33),         # aliasing, 33 maps (the last pair holds one map)
    ("gl", (64, 2048), 63, 63, 2),   # direct N = 1024
    ("gl", (16, 8192), 15, 15, 2),   # direct N = 4096: one map per round, two rounds
    ("hp", 600, 1200, 1200, 2),      # caps up to N = 1198: Bluestein length 4096, two rounds
]


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("case", CASES)
def test_ring_kernel_choices_vs_oracle(oracle_mod, sht, case, mode):
    kind, size, lmax, mmax, nmaps = case
    if kind == "hp":
        og, sg = oracle_mod.healpix_grid(size), sht.healpix(size)
    else:
        og, sg = oracle_mod.gl_grid(*size), sht.gl(*size)
    alm = inputs.batch_alm(lmax, mmax, 500 + lmax, nmaps)
    plan = sht.Plan(sg, lmax, mmax)
    plan.debug_ring_kernel(mode)
    got = plan.alm2map(torch.from_numpy(alm).cuda(), "bf16x6_tc")
    plan.sync()
    got = got.double().cpu().numpy()
    if kind == "hp" and size >= 600:
        rings, _ = inputs.healpix_ring_sample(size, 40, 3, n_large=16, n_smooth_cap=12)
        want = oracle_mod.alm2map(og, lmax, mmax, alm, rings=rings)
    else:
        want = oracle_mod.alm2map(og, lmax, mmax, alm)
    errs = [_rl2(got[b], want[b]) for b in range(nmaps)]
    assert max(errs) < 1e-6, (mode, max(errs))


def test_ring_kernel_choices_agree(sht):
    """The kernels differ only in rounding: maps within FP32 rounding of each other."""
    plan = sht.Plan(sht.healpix(64), 128)
    alm = torch.from_numpy(inputs.batch_alm(128, 128, 77, 4)).cuda()
    outs = []
    for mode in (0, 1, 2):
        plan.debug_ring_kernel(mode)
        outs.append(plan.alm2map(alm, "fp32_tc"))
    plan.sync()
    for o in outs[1:]:
        assert float(torch.linalg.norm(o - outs[0]) / torch.linalg.norm(outs[0])) < 1e-6


@pytest.mark.parametrize("mode", [0, 2])
def test_many_requests_use_the_plans_ring_kernel(sht, mode):
    """The many-request form runs each request's rings on the kernel its plan
    chose, with the per-plan arithmetic: bit for bit the per-plan maps."""
    lmaxs = [64, 100, 130, 33]
    plans = [sht.Plan(sht.healpix(max(1, L // 2)), L) for L in lmaxs]
    for p in plans:
        p.debug_ring_kernel(mode)
    alms = [torch.from_numpy(inputs.gaussian_alm(L, L, (12, i))[0]).cuda() for i, L in enumerate(lmaxs)]
    outs = sht.Multi(plans, "fp32_tc").alm2map(alms)
    torch.cuda.synchronize()
    for p, a, o in zip(plans, alms, outs):
        assert torch.equal(o, p.alm2map(a, "fp32_tc"))


def test_ring_kernel_choice_rejects_bad_mode(sht):
    plan = sht.Plan(sht.healpix(4), 8)
    with pytest.raises(sht.ShtError):
        plan.debug_ring_kernel(3)
