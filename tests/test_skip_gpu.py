"""Evanescent skip of the tensor-core forms: starting each (m, ring block)
work item at its first 64-degree group with a value representable in FP32,
from the stored recurrence state, must give maps bit-identical to running the
recurrence from degree m (the skipped values all round to zero, and the
rescaling by powers of two is exact) -- per call and with the plan-time
Lambda operand, built with the skip on or off."""
import pytest
import torch

from paper_1010_1260_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import sht as s
    s.lib()
    return s


@pytest.mark.parametrize("prec", ["fp32_tc", "bf16x3_tc", "bf16x6_tc"])
def test_skip_bit_identical(sht, prec):
    # nside 64, lmax 160: polar rings with large m start many degrees below FP32 range
    plan = sht.Plan(sht.healpix(64), 160)
    alm = torch.from_numpy(inputs.batch_alm(160, 160, 51, 5)).cuda()
    plan.skip_evanescent(False)
    ref = plan.alm2map(alm, prec)
    plan.sync()
    plan.skip_evanescent(True)
    got = plan.alm2map(alm, prec)
    plan.sync()
    assert torch.equal(got, ref)
    plan.lambda_cache(prec)                      # built with the skip on
    assert torch.equal(plan.alm2map(alm, prec), ref)
    plan.skip_evanescent(False)                  # same operand, every stage read
    assert torch.equal(plan.alm2map(alm, prec), ref)
    plan.lambda_cache(prec, enable=False)
    plan.lambda_cache(prec)                      # built with the skip off
    plan.skip_evanescent(True)
    assert torch.equal(plan.alm2map(alm, prec), ref)
    plan.sync()


def test_skip_bit_identical_full_size(sht):
    """HEALPix nside 1024, lmax 2048, 64 maps (the benchmark's workload)."""
    plan = sht.Plan(sht.healpix(1024), 2048)
    alm = torch.from_numpy(inputs.batch_alm(2048, 2048, 3, 64)).cuda()
    plan.skip_evanescent(False)
    ref = plan.alm2map(alm, "bf16x6_tc")
    plan.sync()
    plan.skip_evanescent(True)
    got = plan.alm2map(alm, "bf16x6_tc")
    plan.sync()
    assert torch.equal(got, ref)
