"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function that include/sht.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(sht_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1010_1260_gb300 import build, sht
    build.build()
    return sht.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("sht_plan", "sht_plan_destroy", "sht_alm2map", "sht_map2alm_adjoint",
                 "sht_alm2map_batch", "sht_map2alm_adjoint_batch", "sht_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_bad_arguments_rejected_on_host(lib):
    from paper_1010_1260_gb300 import sht
    h = ctypes.c_void_p()
    g = sht.healpix(4)._c()
    assert lib.sht_plan(None, 4, 4, ctypes.byref(h)) == sht.SHT_EINVAL
    assert lib.sht_plan(ctypes.byref(g), 4, 5, ctypes.byref(h)) == sht.SHT_EINVAL   # mmax > lmax
    assert lib.sht_plan(ctypes.byref(g), -1, 0, ctypes.byref(h)) == sht.SHT_EINVAL
    assert b"mmax" in lib.sht_last_error()
    bad = sht.GridSpec(7)._c()
    assert lib.sht_plan(ctypes.byref(bad), 4, 4, ctypes.byref(h)) == sht.SHT_EINVAL
    g0 = sht.healpix(0)._c()
    assert lib.sht_plan(ctypes.byref(g0), 4, 4, ctypes.byref(h)) == sht.SHT_EINVAL
    big = sht.healpix(4096)._c()
    assert lib.sht_plan(ctypes.byref(big), 4, 4, ctypes.byref(h)) == sht.SHT_EUNSUPPORTED
    rg = sht.rings([0.5, 4.0], [4, 4], [0.0, 0.0])._c()                       # theta > pi
    assert lib.sht_plan(ctypes.byref(rg), 4, 4, ctypes.byref(h)) == sht.SHT_EINVAL
    assert lib.sht_alm2map_batch(None, 1, None, None, 0, None) == sht.SHT_EINVAL
    assert lib.sht_map2alm_adjoint_batch(None, 1, None, None, 0, None) == sht.SHT_EINVAL
    assert lib.sht_lambda_cache(None, sht.PREC["bf16x6_tc"], 1, None) == sht.SHT_EINVAL
    assert lib.sht_lambda_cache_bytes(None, sht.PREC["bf16x6_tc"]) == 0
    assert lib.sht_autotune(None, sht.PREC["bf16x6_tc"], 4, None) == sht.SHT_EINVAL
    assert lib.sht_tiles(None, None, 0) == sht.SHT_EINVAL
    assert lib.sht_set_tiles(None, None, 0) == sht.SHT_EINVAL
    assert lib.sht_debug_withhold_stage(None, 0) == sht.SHT_EINVAL
    assert lib.sht_debug_ring_kernel(None, 0) == sht.SHT_EINVAL
    assert lib.sht_debug_poison_delta(None) == sht.SHT_EINVAL
    assert lib.sht_multi_debug_poison_delta(None) == sht.SHT_EINVAL
    assert lib.sht_multi_tiles(None, None, 2) == sht.SHT_EINVAL
    assert lib.sht_multi_set_tiles(None, None, 2) == sht.SHT_EINVAL
    assert lib.sht_multi_autotune(None, None, None, None) == sht.SHT_EINVAL
    assert lib.sht_alm2map_host(None, 1, 1, None, None, 0, None) == sht.SHT_EINVAL
    assert lib.sht_alm2map_mpart(None, 1, 1, None, None, 0, None, None, 0, None) == sht.SHT_EINVAL
    assert lib.sht_ring_synth_part(None, 1, 1, None, None, 0, None, None, 0, None) == sht.SHT_EINVAL
    assert lib.sht_ring_lengths(None, None) == sht.SHT_EINVAL
    assert lib.sht_debug_report(None, None) == sht.SHT_EINVAL
    assert lib.sht_alm2map_spin2(None, 1, None, None, None, 0, None) == sht.SHT_EINVAL
    assert lib.sht_skip_evanescent(None, 1) == sht.SHT_EINVAL
    assert lib.sht_map2alm_batch(None, 1, None, None, 0, 0, None) == sht.SHT_EINVAL
    assert lib.sht_set_ring_weights(None, None) == sht.SHT_EINVAL
    assert lib.sht_ring_weights(None, None) == sht.SHT_EINVAL
    assert lib.sht_nalm(None) == 0 and lib.sht_npix(None) == 0
    assert lib.sht_plan_destroy(None) == sht.SHT_OK
