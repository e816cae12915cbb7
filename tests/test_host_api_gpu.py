"""sht_alm2map_host: coefficients in host memory to maps in host memory,
pipelined inside the library (uploads, transforms and downloads of
consecutive batches overlap).  Every step equals sht_alm2map_batch on device
buffers, for the FP64 path and a tensor-core form, with host arrays reused
two steps apart (as a streaming caller does) and with pageable memory."""
import ctypes

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


@pytest.mark.parametrize("prec", ["fp64", "bf16x6_tc"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_pipeline_equals_device_calls(sht, prec, pinned):
    plan = sht.Plan(sht.healpix(32), 64)
    B, nsteps = 3, 5
    srcs = [torch.from_numpy(inputs.batch_alm(64, 64, 700 + k, B)) for k in range(nsteps)]
    if pinned:
        srcs = [a.pin_memory() for a in srcs]
    outs = [torch.zeros((B, plan.npix), dtype=sht.MAP_DTYPE[prec], pin_memory=pinned) for _ in range(2)]
    a_arr = (ctypes.c_void_p * nsteps)(*[a.data_ptr() for a in srcs])
    # outputs reused two steps apart: after the call they hold the last two steps
    m_arr = (ctypes.c_void_p * nsteps)(*[outs[k % 2].data_ptr() for k in range(nsteps)])
    L = sht.lib()
    sht.check(L.sht_alm2map_host(plan.handle, nsteps, B, a_arr, m_arr, sht.PREC[prec],
                                 torch.cuda.current_stream().cuda_stream))
    for k in (nsteps - 2, nsteps - 1):
        want = plan.alm2map(srcs[k].cuda(), prec).cpu()
        assert torch.equal(outs[k % 2], want)


def test_host_pipeline_rejects_bad_arguments(sht):
    L = sht.lib()
    plan = sht.Plan(sht.healpix(4), 8)
    arr = (ctypes.c_void_p * 1)(None)
    assert L.sht_alm2map_host(plan.handle, 1, 1, arr, arr, 0, None) == sht.SHT_EINVAL
    assert L.sht_alm2map_host(plan.handle, -1, 1, arr, arr, 0, None) == sht.SHT_EINVAL
    assert L.sht_alm2map_host(plan.handle, 1, 1, arr, arr, 9, None) == sht.SHT_EINVAL
    assert L.sht_alm2map_host(plan.handle, 0, 1, None, None, 0, None) == sht.SHT_OK
