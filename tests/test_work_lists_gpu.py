"""The balanced work lists of the persistent tensor-core launches against
round robin, on the GPU: the maps are the same bit for bit (every item runs
exactly once, whatever CTA runs it) per call and with the plan-time Lambda
operand, at sizes with many more items than CTAs."""
import pytest
import torch

from paper_1010_1260_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import sht as s
    s.lib()
    return s


@pytest.mark.parametrize("prec", ["fp32_tc", "bf16x6_tc"])
def test_lists_equal_round_robin(sht, prec):
    # nside 128, lmax 256: 2 ring blocks x 257 orders = 514 items for 152 CTAs
    plan = sht.Plan(sht.healpix(128), 256)
    alm = torch.from_numpy(inputs.batch_alm(256, 256, 17, 3)).cuda()
    lists = plan.alm2map(alm, prec)
    plan.sync()
    plan.debug_work_lists(False)
    rr = plan.alm2map(alm, prec)
    plan.sync()
    assert torch.equal(lists, rr)
    plan.lambda_cache(prec)
    cached_rr = plan.alm2map(alm, prec)
    plan.debug_work_lists(True)
    cached_lists = plan.alm2map(alm, prec)
    plan.sync()
    assert torch.equal(cached_rr, lists) and torch.equal(cached_lists, lists)


def test_lists_equal_round_robin_full_size(sht):
    """HEALPix nside 1024, lmax 2048 (16 ring blocks x 2049 orders), 4 maps."""
    plan = sht.Plan(sht.healpix(1024), 2048)
    alm = torch.from_numpy(inputs.batch_alm(2048, 2048, 23, 4)).cuda()
    lists = plan.alm2map(alm, "bf16x6_tc")
    plan.sync()
    plan.debug_work_lists(False)
    rr = plan.alm2map(alm, "bf16x6_tc")
    plan.sync()
    assert torch.equal(lists, rr)
