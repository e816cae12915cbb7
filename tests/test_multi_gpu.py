"""The batching form: many one-map requests of uneven grids and band limits
in one persistent launch (FP64) -- equal to the per-plan path bit for bit,
equal to the oracle, and replayable from a captured CUDA graph."""
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


def _requests(sht, lmaxs):
    plans = [sht.Plan(sht.healpix(max(1, L // 2)), int(L)) for L in lmaxs]
    alms = [torch.from_numpy(inputs.gaussian_alm(int(L), int(L), (4, i))[0]).cuda() for i, L in enumerate(lmaxs)]
    return plans, alms


def test_multi_equals_per_plan_bitwise(sht):
    lmaxs = [64, 75, 130, 33, 200, 64, 97]
    plans, alms = _requests(sht, lmaxs)
    multi = sht.Multi(plans, "fp64")
    outs = multi.alm2map(alms)
    torch.cuda.synchronize()
    for p, a, o in zip(plans, alms, outs):
        assert torch.equal(o, p.alm2map(a))


def test_multi_matches_oracle(oracle_mod, sht):
    lmaxs = [16, 40, 23, 64]
    plans, alms = _requests(sht, lmaxs)
    outs = sht.Multi(plans, "fp64").alm2map(alms)
    torch.cuda.synchronize()
    for L, a, o in zip(lmaxs, alms, outs):
        g = oracle_mod.healpix_grid(max(1, L // 2))
        want = oracle_mod.alm2map(g, L, L, a.cpu().numpy()[None])[0]
        got = o.cpu().numpy()
        assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-10


def test_multi_graph_replay_equals_eager(sht):
    lmaxs = [64, 128, 90, 256]
    plans, alms = _requests(sht, lmaxs)
    multi = sht.Multi(plans, "fp64")
    eager = [o.clone() for o in multi.alm2map(alms)]
    outs = multi.outputs()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        multi.alm2map(alms, outs)          # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    for o in outs:
        o.zero_()
    with torch.cuda.graph(g):
        multi.alm2map(alms, outs)
    for _ in range(3):
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        for o, e in zip(outs, eager):
            assert torch.equal(o, e)


@pytest.mark.parametrize("prec", ["fp32_tc", "bf16x6_tc"])
def test_multi_tensor_core_form(sht, prec):
    """One persistent tensor-core launch over all requests: bit for bit the
    per-plan tensor-core path (same items, same arithmetic), and close to FP64."""
    lmaxs = [64, 100, 48, 130, 33, 200]
    plans, alms = _requests(sht, lmaxs)
    multi = sht.Multi(plans, prec)
    outs = multi.alm2map(alms)
    torch.cuda.synchronize()
    for p, a, o in zip(plans, alms, outs):
        assert torch.equal(o, p.alm2map(a, prec))
        ref = p.alm2map(a).float()
        assert float(torch.linalg.norm(o - ref) / torch.linalg.norm(ref)) < (1e-5 if prec == "fp32_tc" else 1e-6)


def test_multi_tensor_core_launch_count(sht):
    """A tensor-core multi call is a fixed handful of launches whatever the
    number of requests: one operand prep, one Legendre launch, and the ring
    launches (register-FFT kernel and at most two shared-memory ring lists)."""
    lmaxs = inputs.request_lmax(40, 11, 16, 160)
    plans, alms = _requests(sht, lmaxs)
    multi = sht.Multi(plans, "fp32_tc")
    outs = multi.alm2map(alms)
    torch.cuda.synchronize()
    n0 = sht.kernel_launches()
    multi.alm2map(alms, outs)
    torch.cuda.synchronize()
    assert 3 <= sht.kernel_launches() - n0 <= 5


def test_multi_tensor_core_graph_replay(sht):
    lmaxs = [64, 128, 90, 256]
    plans, alms = _requests(sht, lmaxs)
    multi = sht.Multi(plans, "bf16x6_tc")
    eager = [o.clone() for o in multi.alm2map(alms)]
    outs = multi.outputs()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        multi.alm2map(alms, outs)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        multi.alm2map(alms, outs)
    for _ in range(2):
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        for o, e in zip(outs, eager):
            assert torch.equal(o, e)


def test_multi_tensor_core_log_uniform(oracle_mod, sht):
    lmaxs = inputs.request_lmax(256, 4)
    plans, alms = _requests(sht, lmaxs)
    outs = sht.Multi(plans, "fp32_tc").alm2map(alms)
    torch.cuda.synchronize()
    rng = np.random.default_rng(8)
    for i in sorted(set(rng.choice(256, 5, replace=False).tolist()) | {int(np.argmin(lmaxs))}):
        assert torch.equal(outs[i], plans[i].alm2map(alms[i], "fp32_tc"))
    i = int(np.argmin(lmaxs))
    L = int(lmaxs[i])
    g = oracle_mod.healpix_grid(L // 2)
    want = oracle_mod.alm2map(g, L, L, alms[i].cpu().numpy()[None])[0]
    got = outs[i].double().cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-5


def test_multi_log_uniform_requests(oracle_mod, sht):
    """256 requests, lmax log-uniform in [64, 2048], nside = lmax // 2: bit for
    bit equal to the per-plan path on a sample, and to the oracle on the
    smallest request."""
    lmaxs = inputs.request_lmax(256, 4)
    plans, alms = _requests(sht, lmaxs)
    multi = sht.Multi(plans, "fp64")
    outs = multi.alm2map(alms)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    for i in sorted(set(rng.choice(256, 6, replace=False).tolist()) | {int(np.argmin(lmaxs))}):
        assert torch.equal(outs[i], plans[i].alm2map(alms[i]))
    i = int(np.argmin(lmaxs))
    L = int(lmaxs[i])
    g = oracle_mod.healpix_grid(L // 2)
    want = oracle_mod.alm2map(g, L, L, alms[i].cpu().numpy()[None])[0]
    assert np.max(np.abs(outs[i].cpu().numpy() - want)) / np.max(np.abs(want)) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "bf16x6_tc"])
def test_multi_repeated_plan(sht, prec):
    """One plan serving several requests with different coefficients: every
    request's map equals that plan's own transform of its coefficients."""
    p, q = sht.Plan(sht.healpix(32), 64), sht.Plan(sht.healpix(20), 40)
    plans = [p, p, q, p]
    alms = [torch.from_numpy(inputs.gaussian_alm(pl.lmax, pl.lmax, (9, i))[0]).cuda() for i, pl in enumerate(plans)]
    outs = sht.Multi(plans, prec).alm2map(alms)
    torch.cuda.synchronize()
    for pl, a, o in zip(plans, alms, outs):
        assert torch.equal(o, pl.alm2map(a, prec))
    assert not torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", ["fp64", "fp32_tc"])
def test_multi_largest_request_vs_oracle(oracle_mod, sht, prec):
    """The largest of 256 log-uniform requests (lmax 2048, nside 1024) inside a
    multi call, against the oracle on a stratified ring sample."""
    lmaxs = inputs.request_lmax(256, 4)
    i = int(np.argmax(lmaxs))
    L = int(lmaxs[i])
    plans, alms = _requests(sht, lmaxs)
    outs = sht.Multi(plans, prec).alm2map(alms)
    torch.cuda.synchronize()
    nside = L // 2
    rings, _ = inputs.healpix_ring_sample(nside, 24, 5, n_large=6, n_smooth_cap=4)
    want = oracle_mod.alm2map(oracle_mod.healpix_grid(nside), L, L, alms[i].cpu().numpy()[None], rings=rings)[0]
    got = outs[i].double().cpu().numpy()
    ok = np.isfinite(want)
    d = got[ok] - want[ok]
    if prec == "fp64":
        assert np.max(np.abs(d)) / np.max(np.abs(want[ok])) < 1e-10
    else:
        assert np.linalg.norm(d) / np.linalg.norm(want[ok]) < 1e-5


def test_multi_rejects_bad_arguments(sht):
    import ctypes
    L = sht.lib()
    h = ctypes.c_void_p()
    assert L.sht_multi_create(0, None, 0, ctypes.byref(h)) == sht.SHT_EINVAL
    plan = sht.Plan(sht.healpix(4), 8)
    arr = (ctypes.c_void_p * 1)(plan.handle)
    assert L.sht_multi_create(1, arr, 9, ctypes.byref(h)) == sht.SHT_EINVAL
    assert L.sht_multi_alm2map(None, None, None, None) == sht.SHT_EINVAL


@pytest.mark.parametrize("prec", ["fp64", "fp32_tc", "bf16x6_tc"])
def test_multi_tiles_bit_identical_and_autotune(sht, prec):
    """Every tile shape of a multi-request context gives the same maps bit for
    bit; the autotuner keeps one of the candidates."""
    plans, alms = _requests(sht, [64, 130, 33, 200, 97])
    mc = sht.Multi(plans, prec)
    ref = [o.clone() for o in mc.alm2map(alms)]
    torch.cuda.synchronize()
    assert mc.tiles() == {"fp64_ctas_per_sm": 8, "ring_threads": 256}
    cands = [(c, 256) for c in (2, 4, 8, 16)] if prec == "fp64" else [(8, 256), (8, 512)]
    for c, t in cands:
        mc.set_tiles(c, t)
        outs = mc.alm2map(alms)
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert torch.equal(o, r), (c, t)
    tiles = mc.autotune(alms)
    assert (tiles["fp64_ctas_per_sm"], tiles["ring_threads"]) in cands
    outs = mc.alm2map(alms)
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    with pytest.raises(Exception):
        mc.set_tiles(0, 256)
    with pytest.raises(Exception):
        mc.set_tiles(8, 384)
    mc.close()
