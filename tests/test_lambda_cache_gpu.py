"""Plan-time Lambda operand of the tensor-core forms: a launch that streams
the cached tiles must give maps bit-identical to the launch that runs the
FP64 recurrence (same values, same pieces, same tensor-core products in the
same order), and therefore the same error against the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_1010_1260_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp32_tc": 1e-5, "bf16x3_tc": 3e-5, "bf16x6_tc": 1e-6}
FORMS = ["fp32_tc", "bf16x3_tc", "bf16x6_tc"]


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import sht as s
    s.lib()
    return s


def _rl2(got, want):
    ok = np.isfinite(want)  # the oracle leaves rings it did not compute as NaN
    return float(np.linalg.norm(got[ok] - want[ok]) / np.linalg.norm(want[ok]))


def _expected_bytes(npairs, lmax, mmax, prec):
    steps = 16 if prec == "fp32_tc" else 32
    pieces = 3 if prec == "bf16x6_tc" else 2
    nst = sum((lmax - m + steps) // steps for m in range(mmax + 1))
    return nst * ((npairs + 127) // 128) * 2 * pieces * 4096


CASES = [
    ("hp", 16, 40, 40, 3),
    ("hp", 37, 70, 61, 1),      # 74 ring pairs, lmax - m not a multiple of the stage
    ("gl", (128, 256), 127, 127, 2),
    ("hp", 64, 130, 130, 65),   # two launch groups, two ring blocks
]


@pytest.mark.parametrize("prec", FORMS)
@pytest.mark.parametrize("case", CASES)
def test_cached_equals_recurrence(oracle_mod, sht, case, prec):
    kind, size, lmax, mmax, nmaps = case
    if kind == "hp":
        og, sg = oracle_mod.healpix_grid(size), sht.healpix(size)
    else:
        og, sg = oracle_mod.gl_grid(*size), sht.gl(*size)
    alm = inputs.batch_alm(lmax, mmax, 500 + lmax, nmaps)
    a = torch.from_numpy(alm).cuda()
    plan = sht.Plan(sg, lmax, mmax)
    ref = plan.alm2map(a, prec)
    plan.sync()
    npairs = (og["nrings"] + 1) // 2
    assert plan.lambda_cache_bytes(prec) == _expected_bytes(npairs, lmax, mmax, prec)
    plan.lambda_cache(prec)
    got = plan.alm2map(a, prec)
    plan.sync()
    assert torch.equal(got, ref)
    want = oracle_mod.alm2map(og, lmax, mmax, alm)
    g = got.double().cpu().numpy()
    assert max(_rl2(g[b], want[b]) for b in range(nmaps)) < TOL[prec]
    # other forms on the same plan still run the recurrence and are unaffected
    other = "fp32_tc" if prec != "fp32_tc" else "bf16x6_tc"
    o1 = plan.alm2map(a, other)
    plan.lambda_cache(prec, enable=False)
    o2 = plan.alm2map(a, other)
    again = plan.alm2map(a, prec)
    plan.sync()
    assert torch.equal(o1, o2)
    assert torch.equal(again, ref)


def test_cache_api_edges(sht):
    plan = sht.Plan(sht.healpix(8), 20)
    assert plan.lambda_cache_bytes("fp64") == 0
    with pytest.raises(sht.ShtError) as ei:
        plan.lambda_cache("fp64")
    assert ei.value.code == sht.SHT_EINVAL
    plan.lambda_cache("bf16x6_tc")
    plan.lambda_cache("bf16x6_tc")             # present: no-op
    plan.lambda_cache("bf16x6_tc", enable=False)
    plan.lambda_cache("bf16x6_tc", enable=False)  # absent: no-op
    plan.close()                               # frees a cache it may hold
    p2 = sht.Plan(sht.healpix(8), 20)
    p2.lambda_cache("fp32_tc")
    p2.close()


def test_cached_full_size(oracle_mod, sht):
    """HEALPix nside 1024, lmax 2048, 64 maps (the benchmark's workload) in
    the BF16 six-product form: bit-identical to the recurrence launch, and
    maps 0 and 63 against the oracle on sampled rings."""
    og = oracle_mod.healpix_grid(1024)
    plan = sht.Plan(sht.healpix(1024), 2048)
    alm = inputs.batch_alm(2048, 2048, 3, 64)
    a = torch.from_numpy(alm).cuda()
    ref = plan.alm2map(a, "bf16x6_tc")
    plan.sync()
    assert plan.lambda_cache_bytes("bf16x6_tc") == _expected_bytes(2048, 2048, 2048, "bf16x6_tc")
    plan.lambda_cache("bf16x6_tc")
    got = plan.alm2map(a, "bf16x6_tc")
    plan.sync()
    assert torch.equal(got, ref)
    del ref
    rings = inputs.sample_rings(og["nrings"], 8, 41)
    for b in (0, 63):
        want = oracle_mod.alm2map(og, 2048, 2048, alm[b: b + 1], rings=rings)[0]
        g = got[b].double().cpu().numpy()
        assert _rl2(g, want) < TOL["bf16x6_tc"]
    plan.close()
