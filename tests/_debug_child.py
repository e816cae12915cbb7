"""Small transforms through the index-checked debug build of the library
(SHT_LIBRARY points at it; started by tests/test_debug_build_gpu.py): every
form and launch path once, each checked against the oracle, then one JSON line
with the errors and every plan's index-check report."""
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1010_1260_gb300 import inputs, sht  # noqa: E402


def rl2(got, want):
    ok = np.isfinite(want)
    return float(np.linalg.norm(got[ok] - want[ok]) / np.linalg.norm(want[ok]))


def main():
    torch.cuda.set_device(0)
    res = {"library": sht.LIB_PATH, "errors": {}, "reports": {}}
    cases = [("hp16", sht.healpix(16), oracle.healpix_grid(16), 40, 3),
             ("gl", sht.gl(64, 129), oracle.gl_grid(64, 129), 63, 2),
             ("hp64", sht.healpix(64), oracle.healpix_grid(64), 128, 4)]
    plans = []
    for name, g, og, L, B in cases:
        plan = sht.Plan(g, L)
        plans.append((name, plan))
        a = inputs.batch_alm(L, L, 900 + L, B)
        want = oracle.alm2map(og, L, L, a)
        ad = torch.from_numpy(a).cuda()
        got = plan.alm2map(ad).cpu().numpy()
        res["errors"][name + "/fp64"] = rl2(got, want)
        for prec in ("fp32_tc", "bf16x6_tc"):
            for mode in (0, 1, 2):
                plan.debug_ring_kernel(mode)
                got = plan.alm2map(ad, prec)
                plan.sync()
                res["errors"]["%s/%s/mode%d" % (name, prec, mode)] = rl2(got.double().cpu().numpy(), want)
            plan.debug_ring_kernel(0)
            plan.lambda_cache(prec)
            got = plan.alm2map(ad, prec)
            plan.sync()
            res["errors"]["%s/%s/cached" % (name, prec)] = rl2(got.double().cpu().numpy(), want)
            plan.lambda_cache(prec, False)
        y = inputs.gaussian_map(og["npix"], 901, B)
        g_adj = plan.map2alm_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
        w_adj = oracle.map2alm_adjoint(og, L, L, y)
        res["errors"][name + "/adjoint"] = rl2(g_adj.view(np.float64), w_adj.view(np.float64))
        # the tensor-core transpose (BF16x6) from the plan-time Lambda operand
        y32 = y.astype(np.float32)
        plan.lambda_cache("bf16x6_tc")
        g_tc = plan.map2alm_adjoint(torch.from_numpy(y32).cuda(), "bf16x6_tc").cpu().numpy()
        w_tc = oracle.map2alm_adjoint(og, L, L, y32.astype(np.float64))
        res["errors"][name + "/adjoint_tc/bf16x6_tc"] = rl2(g_tc.view(np.float64), w_tc.view(np.float64))
        plan.lambda_cache("bf16x6_tc", False)
        # partitioned transform over 3 parts, exchange by device copies
        mo, ro = sht.partition(L, L, plan.ring_lengths(), 3)
        sizes = sht.exchange_sizes(mo, ro, 3, B)
        sends = [plan.alm2map_mpart(ad, mo, ro, p, 3) for p in range(3)]
        out = torch.zeros((B, plan.npix), dtype=torch.float64, device="cuda")
        for q in range(3):
            recv = torch.cat([sends[p][sum(sizes[p][:q]): sum(sizes[p][:q]) + sizes[p][q]] for p in range(3)])
            plan.ring_synth_part(recv, mo, ro, q, 3, B, out=out)
        res["errors"][name + "/partitioned"] = rl2(out.cpu().numpy(), want)
        bb = inputs.batch_alm(L, L, 950 + L, B)
        qu = plan.alm2map_spin2(ad, torch.from_numpy(bb).cuda()).cpu().numpy()
        qw, uw = oracle.alm2map_spin2(og, L, L, a, bb)
        res["errors"][name + "/spin2/fp64"] = max(rl2(qu[:, 0], qw), rl2(qu[:, 1], uw))
        hosted = plan.alm2map_host_stream([torch.from_numpy(a).pin_memory()] * 3, "bf16x6_tc")
        res["errors"][name + "/host"] = rl2(hosted[-1].double().numpy(), want)
    # the batching form, both kinds, over the three plans
    grids = {c[0]: c[2] for c in cases}
    reqs = [p for _, p in plans]
    alms = [torch.from_numpy(inputs.gaussian_alm(p.lmax, p.lmax, (13, i))[0]).cuda() for i, p in enumerate(reqs)]
    for prec in ("fp64", "fp32_tc"):
        outs = sht.Multi(reqs, prec).alm2map(alms)
        torch.cuda.synchronize()
        for (name, plan), o, a in zip(plans, outs, alms):
            want = oracle.alm2map(grids[name], plan.lmax, plan.lmax, a.cpu().numpy()[None])[0]
            res["errors"]["multi/%s/%s" % (prec, name)] = rl2(o.double().cpu().numpy(), want)
    for name, plan in plans:
        res["reports"][name] = plan.debug_report()
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
