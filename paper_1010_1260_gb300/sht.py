"""Python binding of libsht (ctypes; argument marshalling only).

Every step of the transform runs in the library's CUDA kernels; PyTorch only
provides device memory and the current stream.  There is no CPU fallback: if
the library has not been built, loading it raises.

    from paper_1010_1260_gb300 import sht
    plan = sht.Plan(sht.healpix(512), lmax=1024)
    m = plan.alm2map(alm)            # alm: cuda complex128 [B, nalm] or [nalm]
    g = plan.map2alm_adjoint(m)      # transpose: cuda complex128
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# SHT_LIBRARY selects another build of the library (e.g. the index-checked
# debug build, _build/debug/libsht.so); it must exist like the default.
LIB_PATH = os.environ.get("SHT_LIBRARY") or os.path.join(_HERE, "_build", "libsht.so")

SHT_OK = 0
SHT_EINVAL = -1
SHT_ENOMEM = -2
SHT_ECUDA = -3
SHT_EUNSUPPORTED = -4
SHT_ETIMEOUT = -5

GRID_GL, GRID_HEALPIX, GRID_RINGS = 0, 1, 2
PREC = {"fp64": 0, "fp32_tc": 1, "bf16x3_tc": 2, "bf16x6_tc": 3}
MAP_DTYPE = {"fp64": torch.float64, "fp32_tc": torch.float32, "bf16x3_tc": torch.float32,
             "bf16x6_tc": torch.float32}


class ShtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libsht error %d: %s" % (code, msg))
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nside", ctypes.c_int), ("nrings", ctypes.c_int),
                ("nphi_gl", ctypes.c_int), ("theta", ctypes.c_void_p), ("nphi", ctypes.c_void_p),
                ("phi0", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libsht.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libsht.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            P, I, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
            L.sht_plan.argtypes = [ctypes.POINTER(_Grid), I, I, ctypes.POINTER(P)]
            L.sht_plan_destroy.argtypes = [P]
            for f in ("sht_nalm", "sht_npix"):
                getattr(L, f).argtypes = [P]
                getattr(L, f).restype = ctypes.c_size_t
            for f in ("sht_nrings", "sht_lmax", "sht_mmax"):
                getattr(L, f).argtypes = [P]
                getattr(L, f).restype = I
            L.sht_alm2map.argtypes = [P, V, V, I, V]
            L.sht_map2alm_adjoint.argtypes = [P, V, V, I, V]
            L.sht_alm2map_batch.argtypes = [P, I, V, V, I, V]
            L.sht_map2alm_adjoint_batch.argtypes = [P, I, V, V, I, V]
            L.sht_last_error.restype = ctypes.c_char_p
            L.sht_profile.argtypes = [P, I]
            L.sht_profile_read.argtypes = [P, I, V, V]
            L.sht_sync.argtypes = [P]
            PP = ctypes.POINTER(ctypes.c_void_p)
            L.sht_multi_create.argtypes = [I, PP, I, PP]
            L.sht_multi_alm2map.argtypes = [P, PP, PP, V]
            L.sht_multi_destroy.argtypes = [P]
            L.sht_alm2map_multi.argtypes = [I, PP, PP, PP, I, V]
            L.sht_lambda_cache.argtypes = [P, I, I, V]
            L.sht_lambda_cache_bytes.argtypes = [P, I]
            L.sht_lambda_cache_bytes.restype = ctypes.c_longlong
            L.sht_autotune.argtypes = [P, I, I, V]
            L.sht_tiles.argtypes = [P, ctypes.POINTER(I), I]
            L.sht_set_tiles.argtypes = [P, ctypes.POINTER(I), I]
            L.sht_debug_withhold_stage.argtypes = [P, I]
            L.sht_skip_evanescent.argtypes = [P, I]
            L.sht_debug_work_lists.argtypes = [P, I]
            L.sht_debug_ring_kernel.argtypes = [P, I]
            L.sht_debug_poison_delta.argtypes = [P]
            L.sht_order_limits.argtypes = [P, ctypes.POINTER(I)]
            L.sht_multi_debug_poison_delta.argtypes = [P]
            L.sht_multi_tiles.argtypes = [P, ctypes.POINTER(I), I]
            L.sht_multi_set_tiles.argtypes = [P, ctypes.POINTER(I), I]
            L.sht_multi_autotune.argtypes = [P, PP, PP, V]
            L.sht_alm2map_host.argtypes = [P, I, I, PP, PP, I, V]
            IP = ctypes.POINTER(I)
            L.sht_partition.argtypes = [I, I, I, IP, I, IP, IP]
            L.sht_ring_lengths.argtypes = [P, IP]
            L.sht_alm2map_mpart.argtypes = [P, I, I, IP, IP, I, V, V, I, V]
            L.sht_ring_synth_part.argtypes = [P, I, I, IP, IP, I, V, V, I, V]
            L.sht_debug_report.argtypes = [P, ctypes.POINTER(ctypes.c_ulonglong)]
            L.sht_alm2map_spin2.argtypes = [P, I, V, V, V, I, V]
            L.sht_work_lists.argtypes = [I, ctypes.POINTER(ctypes.c_longlong), I, ctypes.POINTER(I),
                                         ctypes.POINTER(I)]
            L.sht_map2alm.argtypes = [P, V, V, I, I, V]
            L.sht_map2alm_batch.argtypes = [P, I, V, V, I, I, V]
            L.sht_set_ring_weights.argtypes = [P, V]
            L.sht_ring_weights.argtypes = [P, V]
            L.sht_kernel_launches.argtypes = []
            L.sht_kernel_launches.restype = ctypes.c_ulonglong
            for f in ("sht_plan", "sht_plan_destroy", "sht_alm2map", "sht_map2alm_adjoint",
                      "sht_alm2map_batch", "sht_map2alm_adjoint_batch", "sht_profile",
                      "sht_profile_read", "sht_sync", "sht_multi_create", "sht_multi_alm2map",
                      "sht_multi_destroy", "sht_alm2map_multi", "sht_lambda_cache", "sht_autotune",
                      "sht_tiles", "sht_set_tiles", "sht_debug_withhold_stage", "sht_map2alm",
                      "sht_map2alm_batch", "sht_set_ring_weights", "sht_ring_weights", "sht_skip_evanescent",
                      "sht_work_lists", "sht_debug_work_lists", "sht_debug_ring_kernel",
                      "sht_alm2map_host", "sht_partition", "sht_ring_lengths", "sht_alm2map_mpart",
                      "sht_ring_synth_part", "sht_debug_report", "sht_alm2map_spin2", "sht_debug_poison_delta",
                      "sht_multi_debug_poison_delta", "sht_order_limits", "sht_multi_tiles", "sht_multi_set_tiles",
                      "sht_multi_autotune"):
                getattr(L, f).restype = I
            _lib = L
    return _lib


def check(rc: int):
    if rc != SHT_OK:
        raise ShtError(rc, lib().sht_last_error().decode())


STAGES = ("legendre", "ring", "adj_ring", "adj_legendre", "operand_prep")


def work_lists(costs, nlists: int):
    """The library's work lists (sht_work_lists): items served in order to the
    list with the least total cost so far.  Returns (off, items) as int32
    arrays: list b is items[off[b]:off[b + 1]]."""
    import numpy as np
    c = np.ascontiguousarray(np.asarray(costs, dtype=np.int64))
    off = np.zeros(int(nlists) + 1, dtype=np.int32)
    items = np.zeros(max(1, c.size), dtype=np.int32)
    check(lib().sht_work_lists(int(c.size), c.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), int(nlists),
                               off.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               items.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return off, items[:c.size]


def kernel_launches() -> int:
    """Kernels launched by libsht in this process so far."""
    return int(lib().sht_kernel_launches())


# ------------------------------------------------- partitioned transform --
# Algorithm 3: orders split over parts for the Legendre step, one all-to-all
# of Delta, rings split over parts for the ring step (see sht_partition).

def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def partition(lmax: int, mmax: int, nphi, nparts: int):
    """(m_owner, ring_owner) int32 arrays of the library's balanced partition
    (host only, no GPU)."""
    nphi = np.ascontiguousarray(nphi, dtype=np.int32)
    mo = np.zeros(mmax + 1, dtype=np.int32)
    ro = np.zeros(len(nphi), dtype=np.int32)
    check(lib().sht_partition(int(lmax), int(mmax), len(nphi), _ip(nphi), int(nparts), _ip(mo), _ip(ro)))
    return mo, ro


def exchange_sizes(m_owner, ring_owner, nparts: int, nbatch: int):
    """Complex entries of every block of the all-to-all: sizes[p][q] = block
    from part p to part q = |rings of q| x nbatch x |orders of p|."""
    nm = np.bincount(np.asarray(m_owner), minlength=nparts)
    nr = np.bincount(np.asarray(ring_owner), minlength=nparts)
    return [[int(nr[q]) * nbatch * int(nm[p]) for q in range(nparts)] for p in range(nparts)]


def alm2map_distributed(plan: "Plan", alm: torch.Tensor, m_owner, ring_owner, group=None,
                        out: torch.Tensor | None = None) -> torch.Tensor:
    """One FP64 alm2map split over the ranks of a torch.distributed group
    (rank = part): this rank's orders through the Legendre step, one
    all_to_all_single of Delta, this rank's rings through the ring step.
    Returns the maps with this rank's rings filled (other rings untouched)."""
    import torch.distributed as dist
    part, nparts = dist.get_rank(group), dist.get_world_size(group)
    a = alm.reshape(-1, plan.nalm).contiguous()
    B = a.shape[0]
    send = plan.alm2map_mpart(a, m_owner, ring_owner, part, nparts)
    recv = exchange(send, m_owner, ring_owner, B, group)
    return plan.ring_synth_part(recv, m_owner, ring_owner, part, nparts, B, out=out)


def exchange(send: torch.Tensor, m_owner, ring_owner, nbatch: int, group=None) -> torch.Tensor:
    """The all-to-all of Algorithm 3 over a torch.distributed group: this
    rank's send buffer (blocks by destination) in, its receive buffer (blocks
    by source) out; complex128 exchanged as pairs of float64."""
    import torch.distributed as dist
    part, nparts = dist.get_rank(group), dist.get_world_size(group)
    sizes = exchange_sizes(m_owner, ring_owner, nparts, nbatch)
    recv = torch.empty(sum(sizes[p][part] for p in range(nparts)), dtype=torch.complex128, device=send.device)
    dist.all_to_all_single(torch.view_as_real(recv).reshape(-1), torch.view_as_real(send).reshape(-1),
                           output_split_sizes=[2 * sizes[p][part] for p in range(nparts)],
                           input_split_sizes=[2 * sizes[part][q] for q in range(nparts)], group=group)
    return recv


# ------------------------------------------------------------------ grids --

class GridSpec:
    """A ring grid: Gauss-Legendre, HEALPix or caller-given rings."""

    def __init__(self, kind: int, nside: int = 0, nrings: int = 0, nphi_gl: int = 0,
                 theta=None, nphi=None, phi0=None):
        self.kind = kind
        self.nside = nside
        self.nrings = nrings
        self.nphi_gl = nphi_gl
        self.theta = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
        self.nphi = None if nphi is None else np.ascontiguousarray(nphi, dtype=np.int32)
        self.phi0 = None if phi0 is None else np.ascontiguousarray(phi0, dtype=np.float64)

    def _c(self) -> _Grid:
        g = _Grid()
        g.kind, g.nside, g.nrings, g.nphi_gl = self.kind, self.nside, self.nrings, self.nphi_gl
        g.theta = None if self.theta is None else self.theta.ctypes.data
        g.nphi = None if self.nphi is None else self.nphi.ctypes.data
        g.phi0 = None if self.phi0 is None else self.phi0.ctypes.data
        return g


def gl(nrings: int, nphi: int) -> GridSpec:
    return GridSpec(GRID_GL, nrings=nrings, nphi_gl=nphi)


def healpix(nside: int) -> GridSpec:
    return GridSpec(GRID_HEALPIX, nside=nside)


def rings(theta, nphi, phi0) -> GridSpec:
    theta = np.asarray(theta, dtype=np.float64)
    return GridSpec(GRID_RINGS, nrings=len(theta), theta=theta, nphi=nphi, phi0=phi0)


# ------------------------------------------------------------------- plan --

def _stream_ptr(stream) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


class Plan:
    """A libsht plan on the current CUDA device."""

    def __init__(self, grid: GridSpec, lmax: int, mmax: int | None = None):
        L = lib()
        self.grid = grid
        self.lmax = int(lmax)
        self.mmax = int(lmax if mmax is None else mmax)
        h = ctypes.c_void_p()
        g = grid._c()
        check(L.sht_plan(ctypes.byref(g), self.lmax, self.mmax, ctypes.byref(h)))
        self._h = h
        self.nalm = int(L.sht_nalm(h))
        self.npix = int(L.sht_npix(h))
        self.nrings = int(L.sht_nrings(h))
        self.lambda_cached = set()  # tensor-core forms whose plan-time Lambda operand is built

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sht_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alm2map(self, alm: torch.Tensor, prec: str = "fp64", out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
        """Maps of ``alm`` (cuda complex128, [B, nalm] or [nalm])."""
        if not (alm.is_cuda and alm.dtype == torch.complex128):
            raise TypeError("alm must be a CUDA complex128 tensor")
        single = alm.dim() == 1
        a = alm.reshape(-1, self.nalm).contiguous()
        B = a.shape[0]
        if out is None:
            out = torch.empty((B, self.npix), dtype=MAP_DTYPE[prec], device=alm.device)
        elif not (out.is_contiguous() and out.dtype == MAP_DTYPE[prec] and out.numel() == B * self.npix):
            raise TypeError("bad output tensor")
        check(lib().sht_alm2map_batch(self._h, B, a.data_ptr(), out.data_ptr(), PREC[prec],
                                      _stream_ptr(stream)))
        return out.reshape(self.npix) if single else out.reshape(B, self.npix)

    def alm2map_spin2(self, elm: torch.Tensor, blm: torch.Tensor, out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
        """Q and U maps (float64 [B, 2, npix] or [2, npix]) of spin-2 E and B
        coefficients (cuda complex128, [B, nalm] or [nalm]); FP64."""
        for t in (elm, blm):
            if not (t.is_cuda and t.dtype == torch.complex128):
                raise TypeError("E and B must be CUDA complex128 tensors")
        single = elm.dim() == 1
        e = elm.reshape(-1, self.nalm).contiguous()
        b = blm.reshape(-1, self.nalm).contiguous()
        if e.shape != b.shape:
            raise ValueError("E and B differ in shape")
        B = e.shape[0]
        if out is None:
            out = torch.empty((B, 2, self.npix), dtype=torch.float64, device=e.device)
        elif not (out.is_contiguous() and out.dtype == torch.float64 and out.numel() == 2 * B * self.npix):
            raise TypeError("bad output tensor")
        check(lib().sht_alm2map_spin2(self._h, B, e.data_ptr(), b.data_ptr(), out.data_ptr(), PREC["fp64"],
                                      _stream_ptr(stream)))
        return out.reshape(2, self.npix) if single else out.reshape(B, 2, self.npix)

    def map2alm_adjoint(self, maps: torch.Tensor, prec: str = "fp64", out: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
        """Real-linear transpose of alm2map (cuda complex128 result).  The BF16
        tensor-core forms take float32 maps and need the plan-time Lambda
        operand of that form (lambda_cache)."""
        if not (maps.is_cuda and maps.dtype == MAP_DTYPE[prec]):
            raise TypeError("maps must be a CUDA tensor of dtype %s" % MAP_DTYPE[prec])
        single = maps.dim() == 1
        y = maps.reshape(-1, self.npix).contiguous()
        B = y.shape[0]
        if out is None:
            out = torch.empty((B, self.nalm), dtype=torch.complex128, device=maps.device)
        check(lib().sht_map2alm_adjoint_batch(self._h, B, y.data_ptr(), out.data_ptr(), PREC[prec],
                                              _stream_ptr(stream)))
        return out.reshape(self.nalm) if single else out.reshape(B, self.nalm)

    # ------------------------------------------------ partitioned transform --
    def ring_lengths(self) -> np.ndarray:
        out = np.zeros(self.nrings, dtype=np.int32)
        check(lib().sht_ring_lengths(self._h, _ip(out)))
        return out

    def alm2map_mpart(self, alm: torch.Tensor, m_owner, ring_owner, part: int, nparts: int,
                      send: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Legendre step of one part (FP64): the send buffer of the all-to-all
        (complex128, nrings x B x |orders of part|, grouped by destination)."""
        a = alm.reshape(-1, self.nalm).contiguous()
        B = a.shape[0]
        mo = np.ascontiguousarray(m_owner, dtype=np.int32)
        ro = np.ascontiguousarray(ring_owner, dtype=np.int32)
        n = self.nrings * B * int(np.sum(mo == part))
        if send is None:
            send = torch.empty(n, dtype=torch.complex128, device=a.device)
        elif not (send.is_contiguous() and send.dtype == torch.complex128 and send.numel() >= n):
            raise TypeError("bad send buffer")
        check(lib().sht_alm2map_mpart(self._h, B, int(nparts), _ip(mo), _ip(ro), int(part), a.data_ptr(),
                                      send.data_ptr(), PREC["fp64"], _stream_ptr(stream)))
        return send

    def ring_synth_part(self, recv: torch.Tensor, m_owner, ring_owner, part: int, nparts: int, nbatch: int,
                        out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Ring step of one part (FP64) from its receive buffer: the pixels of
        the part's rings in ``out`` (float64 [nbatch, npix])."""
        mo = np.ascontiguousarray(m_owner, dtype=np.int32)
        ro = np.ascontiguousarray(ring_owner, dtype=np.int32)
        if out is None:
            out = torch.zeros((nbatch, self.npix), dtype=torch.float64, device=recv.device)
        check(lib().sht_ring_synth_part(self._h, int(nbatch), int(nparts), _ip(mo), _ip(ro), int(part),
                                        recv.data_ptr(), out.data_ptr(), PREC["fp64"], _stream_ptr(stream)))
        return out

    # ------------------------------------------------- Lambda operand --
    def lambda_cache_bytes(self, prec: str) -> int:
        """Device bytes the plan-time Lambda operand of form ``prec`` needs."""
        return int(lib().sht_lambda_cache_bytes(self._h, PREC[prec]))

    def lambda_cache(self, prec: str, enable: bool = True, stream=None):
        """Build (or free) the plan-time Lambda operand of a tensor-core form;
        later alm2map calls of that form stream it instead of running the
        recurrence, with identical results."""
        check(lib().sht_lambda_cache(self._h, PREC[prec], 1 if enable else 0, _stream_ptr(stream)))
        if enable:
            self.lambda_cached.add(prec)
        else:
            self.lambda_cached.discard(prec)

    # ------------------------------------------------------- tile shapes --
    TILE_NAMES = ("ring_maps_smooth", "ring_maps_bluestein", "ring_threads", "fp64_legendre_maps",
                  "fp64_ring_maps", "fp32_analysis_maps")

    def autotune(self, prec: str, nbatch: int, stream=None) -> dict:
        """Time the tile-shape candidates for form ``prec`` and batches of
        ``nbatch`` maps on this plan and keep the fastest; returns tiles()."""
        check(lib().sht_autotune(self._h, PREC[prec], int(nbatch), _stream_ptr(stream)))
        return self.tiles()

    def tiles(self) -> dict:
        """The plan's current tile shapes."""
        n = len(self.TILE_NAMES)
        out = (ctypes.c_int * n)()
        check(lib().sht_tiles(self._h, out, n))
        return dict(zip(self.TILE_NAMES, list(out)))

    def set_tiles(self, **kw):
        """Set tile shapes by name (see TILE_NAMES); unnamed ones keep their value."""
        cur = self.tiles()
        for k, v in kw.items():
            if k not in cur:
                raise KeyError(k)
            cur[k] = int(v)
        n = len(self.TILE_NAMES)
        vals = (ctypes.c_int * n)(*[cur[k] for k in self.TILE_NAMES])
        check(lib().sht_set_tiles(self._h, vals, n))

    def skip_evanescent(self, enable: bool = True):
        """Tensor-core forms: start work items after their all-zero degrees."""
        check(lib().sht_skip_evanescent(self._h, 1 if enable else 0))

    def debug_withhold_stage(self, stage: int):
        """Test hook: the next tensor-core Legendre launch skips one stage's
        operand copies in its first CTA, so its bounded wait runs out."""
        check(lib().sht_debug_withhold_stage(self._h, int(stage)))

    def debug_work_lists(self, enable: bool):
        """Test hook: False makes the tensor-core launches take their items
        round robin instead of the balanced work lists (same maps)."""
        check(lib().sht_debug_work_lists(self._h, 1 if enable else 0))

    def debug_report(self) -> dict:
        """Index-check report of a debug build (checks_built False in release builds)."""
        out = (ctypes.c_ulonglong * 5)()
        check(lib().sht_debug_report(self._h, out))
        return {"checks_built": bool(out[0]), "violations": int(out[1]), "first_tag": int(out[2]),
                "first_index": int(out[3]), "first_bound": int(out[4])}

    def debug_ring_kernel(self, mode: int):
        """Test hook: FP32 ring-step kernel choice (0 default: register-FFT kernel
        for the Bluestein rings, 1: shared-memory kernel for all rings, 2:
        register-FFT kernel for every ring it can run)."""
        check(lib().sht_debug_ring_kernel(self._h, int(mode)))

    def debug_poison_delta(self):
        """Test hook: fill the plan's Delta workspace with NaN bytes (synchronises)."""
        check(lib().sht_debug_poison_delta(self._h))

    def order_limits(self) -> np.ndarray:
        """Per ring, 1 + the largest order whose FP32 Delta can be nonzero."""
        out = np.zeros(self.nrings, dtype=np.int32)
        check(lib().sht_order_limits(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return out

    # ---------------------------------------------------------- analysis --
    def map2alm(self, maps: torch.Tensor, niter: int = 0, out: torch.Tensor | None = None,
                stream=None, prec: str = "fp64") -> torch.Tensor:
        """Quadrature-weighted analysis of CUDA maps ([B, npix] or [npix];
        float64, float32 for the BF16 tensor-core forms, which need the
        plan-time Lambda operand and niter = 0) with ``niter`` Jacobi
        refinements (complex128 result)."""
        if not (maps.is_cuda and maps.dtype == MAP_DTYPE[prec]):
            raise TypeError("maps must be a CUDA tensor of dtype %s" % MAP_DTYPE[prec])
        single = maps.dim() == 1
        y = maps.reshape(-1, self.npix).contiguous()
        B = y.shape[0]
        if out is None:
            out = torch.empty((B, self.nalm), dtype=torch.complex128, device=maps.device)
        check(lib().sht_map2alm_batch(self._h, B, y.data_ptr(), out.data_ptr(), PREC[prec], int(niter),
                                      _stream_ptr(stream)))
        return out.reshape(self.nalm) if single else out.reshape(B, self.nalm)

    def ring_weights(self) -> np.ndarray:
        """Pixel quadrature weight of every ring."""
        w = np.empty(self.nrings, dtype=np.float64)
        check(lib().sht_ring_weights(self._h, w.ctypes.data))
        return w

    def set_ring_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float64)
        if w.shape != (self.nrings,):
            raise ValueError("need %d weights" % self.nrings)
        check(lib().sht_set_ring_weights(self._h, w.ctypes.data))

    def sync(self):
        """Wait for the plan's device; raise ShtError(SHT_ETIMEOUT) if a kernel
        of this plan gave up a bounded device-side wait."""
        check(lib().sht_sync(self._h))

    # ---------------------------------------------------------- profiling --
    def profile(self, enable: bool = True):
        """Record CUDA events around every kernel this plan launches."""
        check(lib().sht_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{stage: (total ms, launches)} since the last read (synchronises)."""
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        check(lib().sht_profile_read(self._h, n, ms, cnt))
        return {s: (ms[i], cnt[i]) for i, s in enumerate(STAGES)}

    # ------------------------------------------------------- host buffers --
    def alm2map_host(self, alm: torch.Tensor, prec: str = "fp64", out: torch.Tensor | None = None) -> torch.Tensor:
        """alm2map of host coefficients into a host map through the library's
        host-buffer call (one step); pinned host tensors make the copies
        asynchronous."""
        if alm.is_cuda or alm.dtype != torch.complex128:
            raise TypeError("alm must be a host complex128 tensor")
        a = alm.reshape(-1, self.nalm).contiguous()
        if out is None:
            out = torch.empty((a.shape[0], self.npix), dtype=MAP_DTYPE[prec], pin_memory=True)
        return self.alm2map_host_stream([a], prec, outs=[out])[0]

    def alm2map_host_stream(self, alms, prec: str = "fp64", outs=None) -> list:
        """alm2map of a sequence of host batches (complex128, ideally pinned)
        into host maps through the library's pipelined host-buffer call
        (sht_alm2map_host): batch k+1's coefficients go up and batch k-1's maps
        come down while batch k is transformed.  Returns the host maps."""
        alms = [a.reshape(-1, self.nalm) for a in alms]
        if not alms:
            return []
        B = alms[0].shape[0]
        for a in alms:
            if a.is_cuda or a.dtype != torch.complex128 or a.shape[0] != B or not a.is_contiguous():
                raise TypeError("contiguous host complex128 batches of equal size expected")
        if outs is None:
            outs = [torch.empty((B, self.npix), dtype=MAP_DTYPE[prec], pin_memory=True) for _ in alms]
        for o in outs:
            if o.is_cuda or o.dtype != MAP_DTYPE[prec] or o.numel() != B * self.npix or not o.is_contiguous():
                raise TypeError("bad host output tensor")
        n = len(alms)
        a_arr = (ctypes.c_void_p * n)(*[a.data_ptr() for a in alms])
        m_arr = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        check(lib().sht_alm2map_host(self._h, n, B, a_arr, m_arr, PREC[prec], _stream_ptr(None)))
        return outs


class Multi:
    """Many one-map requests of different plans in one call (the batching form)."""

    def __init__(self, plans, prec: str = "fp64"):
        self.plans = list(plans)  # keeps the plans alive
        self.prec = prec
        n = len(self.plans)
        arr = (ctypes.c_void_p * n)(*[p.handle for p in self.plans])
        h = ctypes.c_void_p()
        check(lib().sht_multi_create(n, arr, PREC[prec], ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sht_multi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def debug_poison_delta(self):
        """Test hook: fill the context's Delta workspace with NaN bytes (synchronises)."""
        check(lib().sht_multi_debug_poison_delta(self._h))

    def tiles(self) -> dict:
        """Tile shapes: FP64 persistent CTAs per SM, tensor-core ring-kernel threads."""
        out = (ctypes.c_int * 2)()
        check(lib().sht_multi_tiles(self._h, out, 2))
        return {"fp64_ctas_per_sm": out[0], "ring_threads": out[1]}

    def set_tiles(self, fp64_ctas_per_sm: int, ring_threads: int):
        vals = (ctypes.c_int * 2)(int(fp64_ctas_per_sm), int(ring_threads))
        check(lib().sht_multi_set_tiles(self._h, vals, 2))

    def autotune(self, alms, outs=None, stream=None) -> dict:
        """Time the candidate tile shapes on these requests, keep the fastest; returns tiles()."""
        n = len(self.plans)
        if outs is None:
            outs = self.outputs(alms[0].device)
        a_arr = (ctypes.c_void_p * n)(*[a.data_ptr() for a in alms])
        m_arr = (ctypes.c_void_p * n)(*[m.data_ptr() for m in outs])
        check(lib().sht_multi_autotune(self._h, a_arr, m_arr, _stream_ptr(stream)))
        return self.tiles()

    def outputs(self, device=None):
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        return [torch.empty(p.npix, dtype=MAP_DTYPE[self.prec], device=dev) for p in self.plans]

    def alm2map(self, alms, outs=None, stream=None):
        """alms[i]: cuda complex128 [nalm_i]; returns (or fills) outs[i]: [npix_i]."""
        n = len(self.plans)
        if len(alms) != n:
            raise ValueError("need one coefficient tensor per request")
        for a, p in zip(alms, self.plans):
            if not (a.is_cuda and a.dtype == torch.complex128 and a.is_contiguous() and a.numel() == p.nalm):
                raise TypeError("bad coefficient tensor")
        if outs is None:
            outs = self.outputs(alms[0].device)
        a_arr = (ctypes.c_void_p * n)(*[a.data_ptr() for a in alms])
        m_arr = (ctypes.c_void_p * n)(*[m.data_ptr() for m in outs])
        check(lib().sht_multi_alm2map(self._h, a_arr, m_arr, _stream_ptr(stream)))
        return outs
