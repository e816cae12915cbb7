#!/usr/bin/env python
"""alm2map throughput on GB300: maps/s at lmax = 2048.

Workload (one step): a batch of 64 maps on a HEALPix grid with nside = 1024
(4095 rings, 12,582,912 pixels per map), lmax = mmax = 2048, coefficients
drawn from a Gaussian with C_l = 1 / (l (l + 1)) (seeded, synthetic), one
alm2map of the whole batch through the library's C ABI.  Inputs (2.15 GB of
coefficients) and outputs are larger than the 129 MB L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|fp32_tc|bf16x3_tc]
    python bench.py --impl reference     # the CPU oracle on the same workload

Under torchrun every rank transforms its own batch (weak scaling, no
collective on the data path); the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "alm2map maps/s at lmax=2048 (HEALPix nside 1024, batch of 64 maps)"
UNIT = "maps/s"
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 (profiling recipe): ~2 DFMA/clk/SM x 152 SMs x 2.07 GHz
DTYPE = {"fp64": "f64", "fp32_tc": "f64 recurrence + 3xtf32 MMA, f32 ring step",
         "bf16x3_tc": "f64 recurrence + bf16 hi/lo (3 products) MMA, f32 ring step",
         "bf16x6_tc": "f64 recurrence + bf16 hi/mid/lo (6 products) MMA, f32 ring step"}
# relative-L2 target of each precision form against the FP64 oracle (per map)
TARGET_REL_L2 = {"fp32_tc": 1e-5, "bf16x3_tc": 1e-6, "bf16x6_tc": 1e-6}
TARGET_NOTE = {"bf16x3_tc": "does not meet the 1e-6 relative-L2 target of the split-BF16 form: two 8-bit "
                            "pieces carry about 16 significant bits (measured about 4.9e-6); bf16x6_tc meets it"}
TENSOR_PEAK_RATIO = {"fp32_tc": 0.5, "bf16x3_tc": 1.0, "bf16x6_tc": 1.0}   # tf32 dense = 1/2 bf16 (nominal)
PRODUCTS = {"fp32_tc": 3, "bf16x3_tc": 3, "bf16x6_tc": 6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["fp64", "fp32_tc", "bf16x3_tc", "bf16x6_tc"], default="bf16x6_tc",
                    help="form timed for the headline value (default: split-BF16, 3 pieces, 6 products)")
    ap.add_argument("--fp64-steps", type=int, default=20,
                    help="timed steps of the plain FP64 path on the same batch, median reported (0: skip)")
    ap.add_argument("--nside", type=int, default=1024)
    ap.add_argument("--lmax", type=int, default=2048)
    ap.add_argument("--maps", type=int, default=64)
    ap.add_argument("--cpu-rings", type=int, default=384,
                    help="rings of one map in the CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--acc-rings", type=int, default=64,
                    help="stratified ring sample on which every map of the batch is checked against the oracle")
    ap.add_argument("--acc-full-maps", type=int, default=2,
                    help="maps checked against the oracle on every ring (first and last of the batch)")
    ap.add_argument("--e2e-steps", type=int, default=32,
                    help="steps of the end-to-end (host buffers) measurement, one pipelined call")
    ap.add_argument("--no-clocks", action="store_true", help="do not sample nvidia-smi")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tile shapes")
    ap.add_argument("--lambda-cache", action="store_true",
                    help="tensor-core forms: time the headline with the plan-time Lambda operand")
    ap.add_argument("--no-cached-side", action="store_true",
                    help="tensor-core forms: skip timing the cached-Lambda form beside the headline")
    ap.add_argument("--workload", choices=["batch", "requests"], default="batch",
                    help="batch: 64 maps at lmax 2048 (the headline); requests: 256 one-map requests, "
                         "lmax log-uniform in [64, 2048], nside = lmax // 2, in one multi-request call")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--no-side-forms", action="store_true",
                    help="skip the batching form (256 requests) and the differentiation form (forward + backward) "
                         "timed beside the headline")
    ap.add_argument("--side-steps", type=int, default=3, help="timed steps of each side form")
    ap.add_argument("--side-only", choices=["differentiation", "polarisation", "batching"], default=None,
                    help="run only this side form beside the headline")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x: float, device) -> float:
    """The maximum of x over the ranks of the initialised process group (x
    itself without one): the step time every whole-job figure divides by."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batch_seeds(rank: int, maps: int):
    """Seeds of the maps of one rank's batch: disjoint across ranks (weak scaling)."""
    return [(3, rank * maps + b) for b in range(maps)]


def workload(args):
    return {"workload": "alm2map HEALPix nside=%d lmax=mmax=%d batch=%d" % (args.nside, args.lmax, args.maps),
            "grid": "healpix", "nside": args.nside, "lmax": args.lmax, "mmax": args.lmax,
            "maps_per_gpu": args.maps, "spectrum": "C_l = 1/(l(l+1)) Gaussian, seeds (3, b)",
            "l2": "inputs larger than L2 (alm %.2f GB per step), no flush" % (
                16.0 * (args.lmax + 1) * (args.lmax + 2) / 2 * args.maps / 1e9)}


# --------------------------------------------------------------- CPU oracle --

def cpu_oracle_sample(args, rings_count: int, seed: int = 41):
    """Time the oracle on one map's seeded ring sample; returns (maps/s, seconds, threads, desc)."""
    import oracle
    from paper_1010_1260_gb300 import inputs
    g = oracle.healpix_grid(args.nside)
    alm = inputs.batch_alm(args.lmax, args.lmax, 3, 1)
    rng = np.random.default_rng(seed)
    rings = np.sort(rng.choice(g["nrings"], size=min(rings_count, g["nrings"]), replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    _, nt = oracle.alm2map(g, args.lmax, args.lmax, alm, rings=rings, return_threads=True)
    dt = time.perf_counter() - t0
    frac = len(rings) / g["nrings"]
    maps_per_s = frac / dt
    desc = ("extrapolated: %d of %d rings (seeded uniform sample) of 1 map timed; maps/s = sampled fraction / "
            "time" % (len(rings), g["nrings"]))
    return maps_per_s, dt, nt, desc


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    vals = []
    for _ in range(args.warmup):
        cpu_oracle_sample(args, max(16, args.cpu_rings // 8))
    nt = 0
    desc = ""
    t_tot = 0.0
    for k in range(args.steps):
        v, dt, nt, desc = cpu_oracle_sample(args, args.cpu_rings, seed=41 + k)
        vals.append(v)
        t_tot += dt
    value = statistics.median(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * args.maps / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload(args), "impl": "reference",
            "ms_per_step_note": "extrapolated: %d maps / the sampled maps/s; no step of the whole batch ran" % args.maps,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": desc,
                             "extrapolated": True},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- accuracy --

def _errors(got, want):
    ok = np.isfinite(want)
    d = got[ok] - want[ok]
    return (float(np.max(np.abs(d)) / np.max(np.abs(want[ok]))),
            float(np.linalg.norm(d) / np.linalg.norm(want[ok])))


def check_accuracy(args, alm_h, outs):
    """Per-map error of each form's batch (outs: {form: device maps}) against
    the CPU oracle: every map on a seeded ring sample stratified by ring class
    (poles, equator, belt, cap rings with and without a large prime factor in
    their length), and the first and last map on every ring."""
    import oracle
    from paper_1010_1260_gb300 import inputs
    L, B = args.lmax, alm_h.shape[0]
    g = oracle.healpix_grid(args.nside)
    rings, cls = inputs.healpix_ring_sample(args.nside, args.acc_rings, 77)
    t0 = time.perf_counter()
    want = oracle.alm2map(g, L, L, alm_h, rings=rings)
    full_maps = sorted({0, B - 1})[:max(0, args.acc_full_maps)]
    wf = oracle.alm2map(g, L, L, alm_h[full_maps]) if full_maps else None
    osec = time.perf_counter() - t0
    counts = {}
    for c in cls.values():
        counts[c] = counts.get(c, 0) + 1
    res = {}
    for form, out in outs.items():
        got = out.double().cpu().numpy()
        norm, rl2 = zip(*[_errors(got[b], want[b]) for b in range(B)])
        full = {}
        for i, b in enumerate(full_maps):
            e = _errors(got[b], wf[i])
            full[str(b)] = {"normwise": e[0], "rel_l2": e[1]}
        acc = {"maps_checked": B, "max_normwise": max(norm), "max_rel_l2": max(rl2),
               "per_map_normwise": list(norm), "per_map_rel_l2": list(rl2), "full_maps_all_rings": full}
        if form in TARGET_REL_L2:
            tgt = TARGET_REL_L2[form]
            worst = max(list(rl2) + [v["rel_l2"] for v in full.values()])
            acc.update(target_rel_l2=tgt, meets_target=bool(worst <= tgt))
            if form in TARGET_NOTE:
                acc["note"] = TARGET_NOTE[form]
        else:
            worst = max(list(norm) + [v["normwise"] for v in full.values()])
            acc.update(target_normwise=1e-10, meets_target=bool(worst <= 1e-10))
        res[form] = acc
    head = dict(res[args.prec])
    head.update(rings_checked=[int(r) for r in rings], ring_classes=counts,
                normwise="max|s - s_oracle| / max|s_oracle|", rel_l2="||s - s_oracle|| / ||s_oracle||",
                oracle_seconds=osec, other_forms={k: v for k, v in res.items() if k != args.prec})
    return head


# --------------------------------------------------------------- our impl --

def traffic_for(kernel: str, algorithmic_bytes: float):
    """DRAM bytes per launch of `kernel` at the benchmark's size: the
    measured/algorithmic ratio of a one-kernel ncu capture on a smaller case
    (profiles/traffic.json) times this launch's algorithmic bytes, while the
    kernel's sources are unchanged since the capture (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        tab = json.load(open(path))
    except ValueError:
        return None
    ent = tab.get(kernel)
    if not ent:
        return None
    m = hashlib.sha256()
    for src in ent["sources"]:
        fp = os.path.join(ROOT, src)
        if not os.path.exists(fp):
            return None
        m.update(open(fp, "rb").read())
    if m.hexdigest()[:16] != ent.get("sources_sha256_16"):
        return None
    return ent["ratio"] * algorithmic_bytes


def copy_times(a_host, m_host, reps: int = 3):
    """Context for the end-to-end figure: the host link alone, without the
    transform -- one step's upload, one step's download, and both at once on
    two streams (ms, median of `reps`)."""
    import torch
    da = torch.empty_like(a_host, device="cuda")
    dm = torch.empty_like(m_host, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn):
        out = []
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            out.append((time.perf_counter() - t0) * 1e3)
        return statistics.median(out[1:])

    def up():
        with torch.cuda.stream(s1):
            da.copy_(a_host, non_blocking=True)

    def down():
        with torch.cuda.stream(s2):
            m_host.copy_(dm, non_blocking=True)

    res = {"h2d": timed(up), "d2h": timed(down), "both": timed(lambda: (up(), down()))}
    del da, dm
    return res


def tc_bop_bytes(L: int, M: int, prec: str) -> int:
    """Bytes of the tensor-core B operand image (pieces of C_l a_lm per (m,
    parity) segment, padded to whole stages of KC degrees, 128 columns)."""
    kc = 8 if prec == "fp32_tc" else 16
    kall = sum(2 * (((L - m + 1 + 2 * kc - 1) // (2 * kc)) * kc) for m in range(M + 1))
    pieces, esz = {"fp32_tc": (2, 4), "bf16x3_tc": (2, 2), "bf16x6_tc": (3, 2)}[prec]
    return pieces * 128 * kall * esz


def legendre_flops(R: int, L: int, M: int, B: int, prec: str):
    """Algorithmic flops of one Legendre launch: 3 R N_lm (recurrence) + 4 R N_lm B (contraction)."""
    nlm = (M + 1) * (2 * L + 2 - M) // 2
    return 3.0 * R * nlm + 4.0 * R * nlm * B


def stage_roofline(stage: str, ms: float, args, R: int, lambda_bytes):
    """Roofline of one step's kernel from its CUDA-event time per step."""
    L, B = args.lmax, args.maps
    nlm = (L + 1) * (L + 2) // 2
    nrings = 4 * args.nside - 1
    peaks = _peaks()
    if stage == "ring":
        npix = 12 * args.nside ** 2
        esz = 8 if args.prec == "fp64" else 4
        by = B * (nrings * (L + 1) * 2 * esz + npix * esz)
        ach = by / (ms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        return {"kernel": ("ring_synth (FP64, smooth and Bluestein ring lists)" if args.prec == "fp64" else
                           "FP32 ring step: ring_reg (Bluestein rings) + ring_synth_mf (power-of-two and odd rings)"),
                "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": None if args.prec == "fp64" else traffic_for("ring_step", by),
                "traffic_source": "ncu DRAM bytes of nside 512 / lmax 1024 / 64 maps scaled by algorithmic bytes",
                "bytes_per_step": by, "bytes": "Delta read (complex) + map written", "ms_per_step": ms,
                "peak_source": "MEASURED_PEAKS hbm_gbs"}
    if args.prec == "fp64":
        fl = legendre_flops(R, L, L, B, args.prec)
        ach = fl / (ms * 1e-3) / 1e12
        return {"kernel": "legendre_fwd_fp64", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "nominal FP64 1.25 TFLOP/s (2 DFMA/clk/SM x 152 SMs x 2070 MHz)",
                "flops_per_launch": fl, "ms_per_launch": ms}
    tpk = peaks.get("bf16_tflops_sustained", 1691.3) * TENSOR_PEAK_RATIO[args.prec]
    fl_t = 4.0 * R * nlm * B
    tensor = {"algorithmic_tflops": fl_t / (ms * 1e-3) / 1e12,
              "executed_tflops": PRODUCTS[args.prec] * fl_t / (ms * 1e-3) / 1e12, "peak": tpk,
              "peak_source": "MEASURED_PEAKS bf16 sustained x nominal dtype ratio",
              "frac_executed": PRODUCTS[args.prec] * fl_t / (ms * 1e-3) / 1e12 / tpk}
    if lambda_bytes:
        # cached Lambda operand: streamed once per launch, with a_lm read and Delta written
        by = lambda_bytes + B * (16 * nlm + nrings * (L + 1) * 8)
        ach = by / (ms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        return {"kernel": "legendre_tc_stream (cached Lambda)", "bound": "hbm", "achieved": ach, "peak": peak,
                "unit": "GB/s", "frac": ach / peak, "traffic": traffic_for("legendre_tc_stream", by),
                "traffic_source": "ncu DRAM bytes of nside 512 / lmax 1024 / 64 maps scaled by algorithmic bytes",
                "bytes_per_launch": by, "ms_per_launch": ms, "peak_source": "MEASURED_PEAKS hbm_gbs",
                "bytes": "Lambda operand + a_lm (complex128) + Delta (complex64)", "tensor": tensor}
    # the FP64 recurrence (3 flops per (l, m, ring pair)) bounds the kernel
    fl64 = 3.0 * R * nlm
    ach = fl64 / (ms * 1e-3) / 1e12
    alg_by = tc_bop_bytes(L, L, args.prec) + B * nrings * (L + 1) * 8
    return {"kernel": "legendre_tc", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": traffic_for("legendre_tc", alg_by),
            "algorithmic_bytes": alg_by, "bytes": "B operand image + Delta written",
            "traffic_source": "ncu DRAM bytes of nside 512 / lmax 1024 / 64 maps scaled by algorithmic bytes",
            "peak_source": "nominal FP64 1.25 TFLOP/s (2 DFMA/clk/SM x 152 SMs x 2070 MHz)",
            "flops_per_launch": fl64, "ms_per_launch": ms, "tensor": tensor}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1010_1260_gb300 import build as _build
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1010_1260_gb300 import inputs, sht
    dev = torch.device("cuda", torch.cuda.current_device())
    L, B = args.lmax, args.maps
    plan = sht.Plan(sht.healpix(args.nside), L)
    alm_h = np.empty((B, plan.nalm), dtype=np.complex128)
    for b, seed in enumerate(batch_seeds(rank, B)):
        alm_h[b] = inputs.gaussian_alm(L, L, seed)[0]
    alm = torch.from_numpy(alm_h).to(dev)
    out = torch.empty((B, plan.npix), dtype=sht.MAP_DTYPE[args.prec], device=dev)
    stream = torch.cuda.current_stream()

    tiles = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        tiles = dict(plan.autotune(args.prec, B), seconds=time.perf_counter() - t0)
    lcache = None
    if args.lambda_cache and args.prec != "fp64":
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.lambda_cache(args.prec)
        lcache = {"bytes": plan.lambda_cache_bytes(args.prec), "build_s": time.perf_counter() - t0}

    for _ in range(args.warmup):
        plan.alm2map(alm, args.prec, out=out)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    plan.profile(True)
    plan.profile_read()
    n0 = sht.kernel_launches()
    clk = ClockSampler(local)
    if not args.no_clocks:
        clk.start()
        time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        plan.alm2map(alm, args.prec, out=out)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = sht.kernel_launches() - n0
    stages = plan.profile_read()
    plan.profile(False)
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms_mean = ev[0].elapsed_time(ev[-1]) / args.steps
    ms = statistics.median(step_ms)
    if world > 1:
        ms = max_over_ranks(ms, dev)
        torch.distributed.barrier()
    torch.cuda.synchronize()

    # the plain FP64 GPU path on the same batch, for the headline comparison
    fp64_path = None
    if args.prec != "fp64" and args.fp64_steps > 0:
        out64 = torch.empty((B, plan.npix), dtype=torch.float64, device=dev)
        if not args.no_autotune:
            plan.autotune("fp64", B)
        plan.alm2map(alm, "fp64", out=out64)
        torch.cuda.synchronize()
        fe = [torch.cuda.Event(enable_timing=True) for _ in range(args.fp64_steps + 1)]
        fe[0].record(stream)
        for k in range(args.fp64_steps):
            plan.alm2map(alm, "fp64", out=out64)
            fe[k + 1].record(stream)
        torch.cuda.synchronize()
        t64 = [fe[k].elapsed_time(fe[k + 1]) for k in range(args.fp64_steps)]
        ms64 = max_over_ranks(statistics.median(t64), dev)
        fp64_path = {"value": world * B / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                     "timing": "median of %d steps (CUDA events per step)" % args.fp64_steps,
                     "ms_min_max": [min(t64), max(t64)], "steps": args.fp64_steps,
                     "speedup_of_headline": ms64 / ms}

    # per-map accuracy on a sample of rings against the CPU oracle (rank 0)
    accuracy = None
    if rank == 0 and not args.no_cpu_baseline:
        forms = {args.prec: out}
        if fp64_path is not None:
            forms["fp64"] = out64
        accuracy = check_accuracy(args, alm_h, forms)
        if fp64_path is not None:
            fp64_path["accuracy"] = accuracy["other_forms"].pop("fp64")
    if fp64_path is not None:
        del out64

    # end to end: pinned host coefficients in, host map out, through the binding
    e2e = None
    if args.e2e_steps > 0:
        # through the public API with host buffers: every step uploads its
        # coefficients from pinned memory and downloads its maps; consecutive
        # steps are pipelined (Plan.alm2map_host_stream)
        a_pins = [torch.from_numpy(alm_h).pin_memory() for _ in range(2)]
        m_pins = [torch.empty((B, plan.npix), dtype=sht.MAP_DTYPE[args.prec], pin_memory=True)
                  for _ in range(2)]
        # warm-up through both buffer pairs (device buffers allocated, every
        # pinned page touched once)
        plan.alm2map_host_stream([a_pins[k % 2] for k in range(max(2, args.warmup))], args.prec,
                                 outs=[m_pins[k % 2] for k in range(max(2, args.warmup))])
        torch.cuda.synchronize()
        # three pipelined calls of e2e_steps steps each; the median call (the host
        # link is shared with the node's other GPUs, so single calls vary)
        calls = []
        for _ in range(3):
            t0 = time.perf_counter()
            plan.alm2map_host_stream([a_pins[k % 2] for k in range(args.e2e_steps)], args.prec,
                                     outs=[m_pins[k % 2] for k in range(args.e2e_steps)])
            calls.append((time.perf_counter() - t0) / args.e2e_steps)
        dt = max_over_ranks(statistics.median(calls), dev)
        e2e = {"value": world * B / dt, "unit": UNIT, "h2d_bytes_per_step": int(a_pins[0].numel() * 16),
               "d2h_bytes_per_step": int(m_pins[0].numel() * m_pins[0].element_size()), "ms_per_step": dt * 1000,
               "steps": args.e2e_steps, "pipelined": True, "calls_ms_per_step": [c * 1000 for c in calls],
               "api": "sht_alm2map_host (C ABI: pinned host buffers, copies pipelined inside the library)",
               "copies_alone_ms": copy_times(a_pins[0], m_pins[0])}
        del a_pins, m_pins

    # the same form with the plan-time Lambda operand (the recurrence moved to
    # plan time), timed beside the headline
    cached = None
    if args.prec != "fp64" and not args.lambda_cache and not args.no_cached_side:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.lambda_cache(args.prec)
        build_s = time.perf_counter() - t0
        for _ in range(2):
            plan.alm2map(alm, args.prec, out=out)
        torch.cuda.synchronize()
        plan.profile(True)
        plan.profile_read()
        clk2 = ClockSampler(local)
        if not args.no_clocks:
            clk2.start()
            time.sleep(0.3)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.steps):
            plan.alm2map(alm, args.prec, out=out)
        c1.record(stream)
        torch.cuda.synchronize()
        cclocks = clk2.stop()
        cst = plan.profile_read()
        plan.profile(False)
        cms = c0.elapsed_time(c1) / args.steps
        cms = max_over_ranks(cms, dev)
        cached = {"value": world * B / (cms * 1e-3), "unit": UNIT, "ms_per_step": cms, "steps": args.steps,
                  "stages_ms_per_step": {k: v[0] / args.steps for k, v in cst.items() if v[1]},
                  "lambda_bytes": plan.lambda_cache_bytes(args.prec), "build_s": build_s, "clocks": cclocks,
                  "note": "Lambda computed by the FP64 recurrence once at plan time (sht_lambda_cache), "
                          "streamed from HBM by every call; results bit-identical to the headline's"}
        plan.lambda_cache(args.prec, False)

    # the differentiation and batching forms beside the headline (one GPU)
    side = {}
    if world == 1 and not args.no_side_forms:
        del alm, out
        torch.cuda.empty_cache()
        for name, fn in (("differentiation_form", lambda: measure_differentiation(args, plan, args.side_steps)),
                         ("polarisation_form", lambda: measure_spin2(args, plan, args.side_steps)),
                         ("batching_form", lambda: measure_requests(args, rank, world, args.side_steps, 1))):
            if args.side_only and not name.startswith(args.side_only):
                continue
            try:
                side[name] = fn()
            except Exception as exc:  # reported, not fatal: the headline stands on its own
                side[name] = {"error": "%s: %s" % (type(exc).__name__, exc)}
            torch.cuda.synchronize()
        if "lmaxs" in side.get("batching_form", {}):
            lm = side["batching_form"].pop("lmaxs")
            side["batching_form"]["workload"] = ("%d one-map requests, lmax log-uniform in [64, 2048] (min %d, max %d), "
                                                 "nside = lmax // 2, one multi-request call per step"
                                                 % (args.requests, int(lm.min()), int(lm.max())))

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # roofline of the dominant kernel (and of the other step)
    R = (4 * args.nside - 1 + 1) // 2
    rl = {k: stage_roofline(k, v[0] / args.steps, args, R, lcache["bytes"] if lcache else None)
          for k, v in stages.items() if v[1] and k in ("legendre", "ring")}
    dom = max(rl, key=lambda k: stages[k][0]) if rl else None
    roof = rl.get(dom)
    if "ring" in rl and args.prec != "fp64":
        # the FP32 ring kernels read only the orders below each ring's limit
        # (Delta is exactly zero past it); the algorithmic count keeps every order
        lim = plan.order_limits()
        kept = float(lim.astype(np.float64).sum()) / (lim.size * (L + 1))
        rl["ring"]["delta_orders_read"] = kept
        rl["ring"]["bytes_read_by_kernels"] = int(B * (lim.astype(np.int64).sum() * 8 + 12 * args.nside ** 2 * 4))
    if cached is not None:
        cst = cached["stages_ms_per_step"]
        cached["roofline"] = {k: stage_roofline(k, cst[k], args, R, cached["lambda_bytes"])
                              for k in ("legendre", "ring") if k in cst}

    maps_per_s = world * B / (ms * 1e-3)
    line = {"metric": METRIC, "value": maps_per_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic",
            "config": dict(workload(args), parallelism="replicas x%d" % world, precision=args.prec,
                           lambda_cache=lcache is not None),
            "lambda_cache": lcache, "tiles": tiles, "lambda_cached_form": cached,
            "timing": {"ms_per_step": "median of %d steps (CUDA events per step)" % args.steps,
                       "ms_mean": ms_mean, "ms_min_max": [min(step_ms), max(step_ms)]},
            "roofline": roof, "roofline_other_step": {k: v for k, v in rl.items() if k != dom},
            "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items() if v[1]},
            "gpu_launches": int(launches), "clocks": clocks, "e2e": e2e, "accuracy": accuracy,
            "fp64_path": fp64_path, "differentiation_form": side.get("differentiation_form"),
            "polarisation_form": side.get("polarisation_form"),
            "batching_form": side.get("batching_form")}
    if world == 1 and not args.no_cpu_baseline:
        v, dt, nt, desc = cpu_oracle_sample(args, args.cpu_rings)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": desc,
                                "seconds": dt, "extrapolated": True}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except (OSError, ValueError):
        return {}


def measure_requests(args, rank, world, steps, warmup):
    """The batching form: 256 one-map requests, lmax log-uniform in [64, 2048],
    nside = lmax // 2, in one multi-request call per step; requests/s per form."""
    import torch
    from paper_1010_1260_gb300 import inputs, sht
    t0 = time.perf_counter()
    lmaxs = inputs.request_lmax(args.requests, 4)
    plans = [sht.Plan(sht.healpix(max(1, int(L) // 2)), int(L)) for L in lmaxs]
    alms = [torch.from_numpy(inputs.gaussian_alm(int(L), int(L), (4, rank * args.requests + i))[0]).cuda()
            for i, L in enumerate(lmaxs)]
    res = {"setup_s": time.perf_counter() - t0, "lmaxs": lmaxs}
    stream = torch.cuda.current_stream()
    for prec in ("fp64", "fp32_tc"):
        multi = sht.Multi(plans, prec)
        outs = multi.outputs()
        t1 = time.perf_counter()
        tiles = dict(multi.autotune(alms, outs), seconds=time.perf_counter() - t1)
        for _ in range(warmup):
            multi.alm2map(alms, outs)
        torch.cuda.synchronize()
        n0 = sht.kernel_launches()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for k in range(steps):
            multi.alm2map(alms, outs)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        ms = statistics.median([ev[k].elapsed_time(ev[k + 1]) for k in range(steps)])
        ms = max_over_ranks(ms, torch.device("cuda", torch.cuda.current_device()))
        res[prec] = {"ms_per_step": ms, "requests_per_s": world * args.requests / (ms * 1e-3),
                     "gpu_launches_per_step": (sht.kernel_launches() - n0) / steps, "tiles": tiles,
                     "timing": "median of %d steps (CUDA events per step)" % steps}
        multi.close()
        del outs
    res["total_alm"] = int(sum(p.nalm for p in plans))
    res["total_pixels"] = int(sum(p.npix for p in plans))
    del alms, plans
    torch.cuda.empty_cache()
    return res


def measure_differentiation(args, plan, steps):
    """The differentiation form: B = 16 maps at the headline's grid and band
    limit, loss = sum_p w_p (s_p - d_p)^2 through the autograd op: forward in
    FP64 and in the headline's form with the FP64 transpose as backward, and
    (BF16 forms) forward from the plan-time Lambda operand with the tensor-core
    transpose of the same form as backward."""
    import torch
    from paper_1010_1260_gb300 import autograd, inputs
    B = 16
    dev = torch.device("cuda", torch.cuda.current_device())
    a0 = torch.from_numpy(inputs.batch_alm(args.lmax, args.lmax, 5, B)).to(dev)
    w, d = inputs.loss_weights(plan.npix, 5, B)
    w = torch.from_numpy(w).to(dev)
    d = torch.from_numpy(d).to(dev)
    stream = torch.cuda.current_stream()
    out = {"maps": B, "loss": "sum_p w_p (s_p - d_p)^2, w ~ U(0.5, 1.5), d ~ N(0, 1), seed 5"}
    had_cache = args.prec in plan.lambda_cached
    variants = [("fp64", False)]
    if args.prec != "fp64" and not had_cache:
        variants.append((args.prec, False))
    if args.prec in ("bf16x6_tc", "bf16x3_tc"):
        variants.append((args.prec, True))
    for fwd, cached in variants:
        if cached and not had_cache:
            t0 = time.perf_counter()
            plan.lambda_cache(fwd)
            out["lambda_build_s"] = time.perf_counter() - t0

        def step():
            a = a0.clone().requires_grad_(True)
            s = autograd.alm2map(a, plan, fwd)
            loss = (w * (s.double() - d) ** 2).sum()
            loss.backward()
            return a.grad
        step()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for k in range(steps):
            step()
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        ms = statistics.median([ev[k].elapsed_time(ev[k + 1]) for k in range(steps)])
        tc_bwd = fwd in ("bf16x6_tc", "bf16x3_tc") and fwd in plan.lambda_cached
        key = "forward_" + fwd + ("_cached_tc_backward" if cached else "")
        out[key] = {"ms_forward_backward": ms, "maps_per_s": B / (ms * 1e-3), "steps": steps,
                    "backward": ("%s tensor-core transpose (FP32 ring analysis + contraction over ring pairs "
                                 "from the Lambda operand)" % fwd) if tc_bwd else
                    "fp64 transpose (ring analysis + Legendre accumulation)"}
        if cached and not had_cache:
            plan.lambda_cache(fwd, False)
    del a0, w, d
    torch.cuda.empty_cache()
    return out


def measure_spin2(args, plan, steps):
    """The polarisation (spin-2) synthesis, FP64: 4 maps of E and B at the
    headline's grid and band limit into Q and U, median of `steps` calls."""
    import torch
    from paper_1010_1260_gb300 import inputs
    B = 4
    dev = torch.device("cuda", torch.cuda.current_device())
    e = torch.from_numpy(inputs.batch_alm(args.lmax, args.lmax, 61, B)).to(dev)
    b = torch.from_numpy(inputs.batch_alm(args.lmax, args.lmax, 62, B)).to(dev)
    out = torch.empty((B, 2, plan.npix), dtype=torch.float64, device=dev)
    plan.alm2map_spin2(e, b, out=out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for k in range(steps):
        plan.alm2map_spin2(e, b, out=out)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.median([ev[k].elapsed_time(ev[k + 1]) for k in range(steps)])
    del e, b, out
    torch.cuda.empty_cache()
    return {"maps": B, "ms_per_call": ms, "qu_maps_per_s": B / (ms * 1e-3), "steps": steps, "dtype": "f64",
            "workload": "E, B Gaussian (C_l = 1/(l(l+1))) -> Q, U on the headline grid"}


def run_requests(args):
    """The batching form: many uneven one-map requests per call (replicas under torchrun)."""
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1010_1260_gb300 import build as _build
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    res = measure_requests(args, rank, world, args.steps, args.warmup)
    lmaxs = res.pop("lmaxs")
    if rank == 0:
        line = {"metric": "alm2map requests/s (256 one-map requests, lmax log-uniform [64, 2048], nside = lmax // 2)",
                "value": res["fp64"]["requests_per_s"], "unit": "requests/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["fp64"]["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "batching form: %d requests" % args.requests,
                           "lmax_min": int(lmaxs.min()), "lmax_max": int(lmaxs.max()),
                           "total_alm": res["total_alm"], "total_pixels": res["total_pixels"]},
                "forms": res}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "requests":
        return run_requests(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
