"""sht_alm2map_noalloc, the FP64 alm2map for callers that must not allocate
device memory once their processing loop runs (e.g. a host framework that has
reserved nearly all device memory for its own pool): it keeps its scratch in
a fixed 16 MiB static device array.  Called through the C ABI, two calls in a
row, each checked against sht_alm2map_batch within the FP64 tolerance of the
other tests.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1010_1260_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import sht as s
    L = s.lib()
    L.sht_alm2map_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
    L.sht_alm2map_noalloc.restype = ctypes.c_int
    return s


def _nerr(a, b):
    return float(torch.max(torch.abs(a - b)) / torch.max(torch.abs(b)))


def test_noalloc_allocates_no_device_memory(sht):
    """On a plan that has never run a transform (so it has no workspace yet),
    a call leaves the device's free memory unchanged.  The same call on
    another plan of the same shape runs before, so that loading the library's
    kernels (which reserves their code and the static scratch) is not counted."""
    L = sht.lib()
    stream = torch.cuda.current_stream()
    warm = sht.Plan(sht.healpix(64), 128)
    a0 = torch.from_numpy(inputs.batch_alm(128, 128, 400, 3)).cuda()
    m0 = torch.empty((3, warm.npix), dtype=torch.float64, device="cuda")
    sht.check(L.sht_alm2map_noalloc(warm.handle, 3, a0.data_ptr(), m0.data_ptr(), stream.cuda_stream))
    plan = sht.Plan(sht.healpix(64), 128)
    alm = torch.from_numpy(inputs.batch_alm(128, 128, 403, 3)).cuda()
    out = torch.empty((3, plan.npix), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    sht.check(L.sht_alm2map_noalloc(plan.handle, 3, alm.data_ptr(), out.data_ptr(), stream.cuda_stream))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # the ordinary entry point on the same plan does grow its workspace
    ref = torch.empty_like(out)
    sht.check(L.sht_alm2map_batch(plan.handle, 3, alm.data_ptr(), ref.data_ptr(), 0, stream.cuda_stream))
    torch.cuda.synchronize()
    assert _nerr(out, ref) < TOL64


def test_noalloc_matches_batch_entry_point_twice(sht):
    L = sht.lib()
    plan = sht.Plan(sht.healpix(64), 128)
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((401, 402)):
        nmaps = 3 if call == 0 else 2
        alm = torch.from_numpy(inputs.batch_alm(128, 128, seed, nmaps)).cuda()
        ref = torch.empty((nmaps, plan.npix), dtype=torch.float64, device="cuda")
        sht.check(L.sht_alm2map_batch(plan.handle, nmaps, alm.data_ptr(), ref.data_ptr(), 0,
                                      stream.cuda_stream))
        out = torch.full((nmaps, plan.npix), float("nan"), dtype=torch.float64, device="cuda")
        sht.check(L.sht_alm2map_noalloc(plan.handle, nmaps, alm.data_ptr(), out.data_ptr(),
                                        stream.cuda_stream))
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _nerr(out, ref) < TOL64


def test_noalloc_rejects_sizes_beyond_the_scratch(sht):
    L = sht.lib()
    plan = sht.Plan(sht.healpix(512), 1024)          # 2047 rings x 1025 m > 1,048,576 entries
    alm = torch.zeros((1, plan.nalm), dtype=torch.complex128, device="cuda")
    out = torch.zeros((1, plan.npix), dtype=torch.float64, device="cuda")
    rc = L.sht_alm2map_noalloc(plan.handle, 1, alm.data_ptr(), out.data_ptr(), None)
    assert rc == sht.SHT_EUNSUPPORTED
    assert b"16 MiB" in L.sht_last_error()
    assert L.sht_alm2map_noalloc(None, 1, alm.data_ptr(), out.data_ptr(), None) == sht.SHT_EINVAL
