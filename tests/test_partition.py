"""The partitioned transform's host side (Algorithm 3, no GPU): the balanced
partition of orders and rings, and the all-to-all exchange of Delta between
two gloo ranks on the CPU in the layouts include/sht.h documents."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import build, sht as s
    build.build()
    s.lib()
    return s


def _healpix_nphi(nside):
    return np.array([4 * min(i, nside, 4 * nside - i) for i in range(1, 4 * nside)], dtype=np.int32)


@pytest.mark.parametrize("nparts", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("lmax,mmax,nside", [(2048, 2048, 1024), (100, 60, 32), (9, 9, 2)])
def test_partition_is_balanced(sht, nparts, lmax, mmax, nside):
    nphi = _healpix_nphi(nside)
    mo, ro = sht.partition(lmax, mmax, nphi, nparts)
    assert mo.shape == (mmax + 1,) and ro.shape == (len(nphi),)
    assert mo.min() >= 0 and mo.max() < nparts and ro.min() >= 0 and ro.max() < nparts
    for m in range(mmax + 1):            # pairs (m, mmax - m) stay together
        assert mo[m] == mo[mmax - m]
    work = np.bincount(mo, weights=lmax - np.arange(mmax + 1) + 1, minlength=nparts)
    pair = 2 * (lmax + 1) - mmax
    assert work.max() - work.min() <= pair
    assert np.all(np.diff(ro) >= 0)        # contiguous ring ranges
    pix = np.bincount(ro, weights=nphi, minlength=nparts)
    assert pix.max() - pix.min() <= 2 * nphi.max()


def test_partition_rejects_bad_arguments(sht):
    L = sht.lib()
    assert L.sht_partition(4, 5, 3, None, 2, None, None) == sht.SHT_EINVAL
    with pytest.raises(sht.ShtError):
        sht.partition(4, 4, [4, 0, 4], 2)


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("nproc", [2, 3])
def test_gloo_exchange_of_delta(sht, nproc):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", str(nproc),
           "--master-addr", "127.0.0.1", "--master-port", str(_port()), os.path.join("tests", "_partition_child.py")]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][0])
    assert out["world"] == nproc
    assert all(x["ok"] for x in out["ranks"]), out
    assert sum(x["orders"] for x in out["ranks"]) == 22
