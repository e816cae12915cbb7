"""The partitioned transform (Algorithm 3) on one GPU: the parts' Legendre
steps, the all-to-all emulated by device copies between the parts' buffers
in the documented layouts, and the parts' ring steps assemble maps equal to
the unpartitioned FP64 alm2map bit for bit (every part runs the same
arithmetic per order and ring); the maps also match the oracle."""
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


def _partitioned(sht, plan, alm, nparts):
    B = alm.shape[0]
    mo, ro = sht.partition(plan.lmax, plan.mmax, plan.ring_lengths(), nparts)
    sizes = sht.exchange_sizes(mo, ro, nparts, B)
    sends = [plan.alm2map_mpart(alm, mo, ro, p, nparts) for p in range(nparts)]
    out = torch.full((B, plan.npix), float("nan"), dtype=torch.float64, device="cuda")
    for q in range(nparts):
        # the block p -> q sits after p's blocks for destinations 0 .. q-1
        blocks = []
        for p in range(nparts):
            o = sum(sizes[p][:q])
            blocks.append(sends[p][o: o + sizes[p][q]])
        recv = torch.cat(blocks)
        plan.ring_synth_part(recv, mo, ro, q, nparts, B, out=out)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("nparts", [1, 2, 3, 4])
@pytest.mark.parametrize("grid,lmax,mmax,nmaps", [("hp16", 40, 40, 3), ("gl", 63, 50, 2), ("hp64", 128, 128, 1)])
def test_partitioned_equals_whole_transform(sht, nparts, grid, lmax, mmax, nmaps):
    g = {"hp16": sht.healpix(16), "hp64": sht.healpix(64), "gl": sht.gl(64, 129)}[grid]
    plan = sht.Plan(g, lmax, mmax)
    alm = torch.from_numpy(inputs.batch_alm(lmax, mmax, 800 + lmax, nmaps)).cuda()
    want = plan.alm2map(alm)
    got = _partitioned(sht, plan, alm, nparts)
    assert torch.isfinite(got).all()
    assert torch.equal(got, want)


def test_partitioned_full_size_vs_oracle(oracle_mod, sht):
    """nside 1024, lmax 2048, 2 maps over 4 parts: equal to the whole FP64
    transform, and to the oracle on a stratified ring sample."""
    plan = sht.Plan(sht.healpix(1024), 2048)
    alm_h = inputs.batch_alm(2048, 2048, 3, 2)
    alm = torch.from_numpy(alm_h).cuda()
    got = _partitioned(sht, plan, alm, 4)
    assert torch.equal(got, plan.alm2map(alm))
    rings, _ = inputs.healpix_ring_sample(1024, 16, 4, n_large=4, n_smooth_cap=4)
    want = oracle_mod.alm2map(oracle_mod.healpix_grid(1024), 2048, 2048, alm_h, rings=rings)
    g = got.cpu().numpy()
    for b in range(2):
        ok = np.isfinite(want[b])
        assert np.max(np.abs(g[b, ok] - want[b, ok])) / np.max(np.abs(want[b, ok])) < 1e-10


def test_partitioned_rejects_other_forms_and_bad_owners(sht):
    plan = sht.Plan(sht.healpix(4), 8)
    alm = torch.zeros((1, plan.nalm), dtype=torch.complex128, device="cuda")
    mo, ro = sht.partition(8, 8, plan.ring_lengths(), 2)
    import ctypes
    L = sht.lib()
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    buf = torch.zeros(4096, dtype=torch.complex128, device="cuda")
    assert L.sht_alm2map_mpart(plan.handle, 1, 2, ip(mo), ip(ro), 0, alm.data_ptr(), buf.data_ptr(),
                               sht.PREC["bf16x6_tc"], None) == sht.SHT_EUNSUPPORTED
    bad = mo.copy()
    bad[0] = 5
    assert L.sht_alm2map_mpart(plan.handle, 1, 2, ip(bad), ip(ro), 0, alm.data_ptr(), buf.data_ptr(), 0,
                               None) == sht.SHT_EINVAL
    assert L.sht_ring_synth_part(plan.handle, 1, 2, ip(mo), ip(ro), 2, buf.data_ptr(), buf.data_ptr(), 0,
                                 None) == sht.SHT_EINVAL
