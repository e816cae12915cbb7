"""Failure detection without a GPU fault.  Every wait of the tensor-core
Legendre kernels is bounded (2 s); the test hook makes the first CTA skip the
operand copies of one stage, so the MMA warp's wait for it runs out.  The CTA
must take its abort path (drain what it issued, free tensor memory, set the
plan's status word), sht_sync must report SHT_ETIMEOUT once, and the plan and
the CUDA context must stay usable: the next call gives the same maps as before."""
import time

import pytest
import torch

from paper_1010_1260_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import sht as s
    s.lib()
    return s


@pytest.mark.parametrize("cached", [False, True])
@pytest.mark.parametrize("prec", ["bf16x6_tc", "fp32_tc"])
def test_bounded_wait_runs_out_and_is_reported(sht, prec, cached):
    plan = sht.Plan(sht.healpix(16), 40)   # 41 work items of 2 stages (BF16) or 3 (TF32)
    alm = torch.from_numpy(inputs.batch_alm(40, 40, 31, 3)).cuda()
    if cached:
        plan.lambda_cache(prec)
    ref = plan.alm2map(alm, prec)
    plan.sync()
    plan.debug_withhold_stage(1)
    t0 = time.time()
    plan.alm2map(alm, prec)
    with pytest.raises(sht.ShtError) as ei:
        plan.sync()
    assert ei.value.code == sht.SHT_ETIMEOUT
    assert time.time() - t0 < 30
    plan.sync()                            # reported once, then cleared
    again = plan.alm2map(alm, prec)        # the hook applied to one launch only
    plan.sync()
    assert torch.equal(again, ref)


def test_hook_argument_checked(sht):
    plan = sht.Plan(sht.healpix(4), 8)
    with pytest.raises(sht.ShtError) as ei:
        plan.debug_withhold_stage(-2)
    assert ei.value.code == sht.SHT_EINVAL
    plan.debug_withhold_stage(-1)          # clears: a normal launch follows
    out = plan.alm2map(torch.from_numpy(inputs.batch_alm(8, 8, 32, 1)).cuda(), "bf16x6_tc")
    plan.sync()
    assert torch.isfinite(out).all()
