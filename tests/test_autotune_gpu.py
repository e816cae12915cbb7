"""Tile shapes and the autotuner: every candidate tile shape gives maps
bit-identical to the default one (the kernels round every product and fused
multiply-add explicitly, so the launch shape cannot change the arithmetic),
and the autotuner's choice is one of the candidates."""
import itertools

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


def test_tc_ring_tiles_bit_identical(sht):
    # HEALPix nside 48: smooth and Bluestein rings; 37 maps: ragged last map group
    plan = sht.Plan(sht.healpix(48), 100)
    alm = torch.from_numpy(inputs.batch_alm(100, 100, 21, 37)).cuda()
    ref = plan.alm2map(alm, "bf16x6_tc")
    plan.sync()
    for gs, gb, nt in itertools.product((1, 2, 4), (1, 2), (256, 512)):
        plan.set_tiles(ring_maps_smooth=gs, ring_maps_bluestein=gb, ring_threads=nt)
        got = plan.alm2map(alm, "bf16x6_tc")
        plan.sync()
        assert torch.equal(got, ref), (gs, gb, nt)


def test_fp64_tiles_bit_identical(sht):
    plan = sht.Plan(sht.healpix(16), 40)
    alm = torch.from_numpy(inputs.batch_alm(40, 40, 22, 11)).cuda()
    ref = plan.alm2map(alm, "fp64")
    plan.sync()
    for bc, g in itertools.product((1, 2, 4, 8), (1, 2, 4, 8, 16)):
        plan.set_tiles(fp64_legendre_maps=bc, fp64_ring_maps=g)
        got = plan.alm2map(alm, "fp64")
        plan.sync()
        assert torch.equal(got, ref), (bc, g)


@pytest.mark.parametrize("prec", ["fp64", "bf16x6_tc"])
def test_autotune_picks_a_candidate_and_keeps_results(oracle_mod, sht, prec):
    og = oracle_mod.healpix_grid(32)
    plan = sht.Plan(sht.healpix(32), 64)
    alm_np = inputs.batch_alm(64, 64, 23, 9)
    alm = torch.from_numpy(alm_np).cuda()
    ref = plan.alm2map(alm, prec)
    plan.sync()
    t = plan.autotune(prec, 9)
    assert t["ring_maps_smooth"] in (1, 2, 4) and t["ring_maps_bluestein"] in (1, 2)
    assert t["ring_threads"] in (256, 512) and t["fp64_legendre_maps"] in (1, 2, 4, 8)
    assert t["fp64_ring_maps"] in (1, 2, 4, 8, 16)
    got = plan.alm2map(alm, prec)
    plan.sync()
    assert torch.equal(got, ref)
    want = oracle_mod.alm2map(og, 64, 64, alm_np)
    g = got.double().cpu().numpy()
    tol = 1e-10 if prec == "fp64" else 1e-6
    for b in range(9):
        err = np.max(np.abs(g[b] - want[b])) / np.max(np.abs(want[b])) if prec == "fp64" else \
            np.linalg.norm(g[b] - want[b]) / np.linalg.norm(want[b])
        assert err < tol


def test_set_tiles_rejects_non_candidates(sht):
    plan = sht.Plan(sht.healpix(8), 16)
    with pytest.raises(sht.ShtError) as ei:
        plan.set_tiles(ring_threads=300)
    assert ei.value.code == sht.SHT_EINVAL
    with pytest.raises(sht.ShtError):
        plan.set_tiles(fp64_legendre_maps=3)
