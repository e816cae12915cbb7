"""Order limits of the tensor-core forms' Delta (a consequence of the
evanescent skip): past a ring's last order with a recurrence value in the FP32
range, Delta_m of that ring is exactly zero, so the Legendre launches leave
those (m, ring block) items out and the FP32 ring kernels read only the orders
below the limit.

  * The limits against the oracle's lambda_lm: at the limit every value of the
    ring is tiny, one order below it some value is not.
  * Maps with the limits equal the maps with the skip off (every item run,
    every order read) bit for bit, after the Delta workspace has been filled
    with NaN bytes, so that a kernel reading an unwritten entry would show --
    every ring kernel choice, per call, cached Lambda operand, the batching
    form, and the full-size workload.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1010_1260_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import sht as s
    s.lib()
    return s


def _nalm(L, M):
    return (M + 1) * (2 * L + 2 - M) // 2


def test_limits_against_oracle(sht):
    nside, L = 64, 160
    plan = sht.Plan(sht.healpix(nside), L)
    lim = plan.order_limits()
    g = oracle.healpix_grid(nside)
    assert lim.shape == (g["nrings"],)
    assert np.all((lim >= 1) & (lim <= L + 1))
    assert np.array_equal(lim, lim[::-1])           # mirrored rings share the pair's limit
    assert lim[0] < L + 1                           # the polar rings do have a limit
    for r in (0, 1, 3, 10, 40, 63, 100, 127):
        lam = np.abs(oracle.lam(L, L, g["x"][r], g["st"][r]))
        m = int(lim[r])
        if m <= L:                                  # every value at the limit is tiny
            off = m * (2 * L + 3 - m) // 2
            assert lam[off: off + L + 1 - m].max() < 2.0 ** -100, (r, m)
        m -= 1                                      # one order below: some value is not
        off = m * (2 * L + 3 - m) // 2
        assert lam[off: off + L + 1 - m].max() > 2.0 ** -160, (r, m)


def _ref_and_plan(sht, nside, L, B, seed):
    plan = sht.Plan(sht.healpix(nside), L)
    alm = torch.from_numpy(inputs.batch_alm(L, L, seed, B)).cuda()
    return plan, alm


@pytest.mark.parametrize("prec", ["fp32_tc", "bf16x6_tc"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_limits_bit_identical_poisoned(sht, prec, mode):
    plan, alm = _ref_and_plan(sht, 64, 160, 5, 61)
    plan.debug_ring_kernel(mode)
    plan.skip_evanescent(False)
    ref = plan.alm2map(alm, prec)
    plan.sync()
    assert torch.isfinite(ref).all()
    plan.skip_evanescent(True)
    plan.debug_poison_delta()
    got = plan.alm2map(alm, prec)
    plan.sync()
    assert torch.equal(got, ref)
    plan.lambda_cache(prec)
    plan.debug_poison_delta()
    got = plan.alm2map(alm, prec)
    plan.sync()
    assert torch.equal(got, ref)
    plan.lambda_cache(prec, enable=False)


def test_limits_multi_poisoned(sht):
    plans = [sht.Plan(sht.healpix(n), L) for n, L in ((16, 40), (64, 160), (32, 80), (64, 128))]
    alms = [torch.from_numpy(inputs.gaussian_alm(p.lmax, p.lmax, (71, i))[0]).cuda() for i, p in enumerate(plans)]
    for prec in ("fp32_tc", "bf16x6_tc"):
        for p in plans:
            p.skip_evanescent(False)
        refs = [p.alm2map(a[None], prec)[0] for p, a in zip(plans, alms)]
        torch.cuda.synchronize()
        for p in plans:
            p.skip_evanescent(True)
        mc = sht.Multi(plans, prec)
        mc.alm2map(alms)                            # allocate and run once
        mc.debug_poison_delta()
        outs = mc.alm2map(alms)
        torch.cuda.synchronize()
        for o, r in zip(outs, refs):
            assert torch.equal(o, r)
        mc.close()


def test_limits_full_size(sht):
    """HEALPix nside 1024, lmax 2048, 64 maps, BF16x6 (the benchmark's workload)."""
    plan, alm = _ref_and_plan(sht, 1024, 2048, 64, 3)
    lim = plan.order_limits()
    kept = float(lim.sum()) / (lim.size * 2049)
    assert 0.5 < kept < 0.9                         # the caps need far fewer orders
    plan.skip_evanescent(False)
    ref = plan.alm2map(alm, "bf16x6_tc")
    plan.sync()
    plan.skip_evanescent(True)
    plan.debug_poison_delta()
    got = plan.alm2map(alm, "bf16x6_tc")
    plan.sync()
    assert torch.equal(got, ref)
