"""Benchmark: solve throughput of the RSD-preconditioned FP64 PCG on one GB300.

One step = one pass of the whole path on resident inputs: rsd_setup (analysis of the
sub-domain tree and interface sets, front assembly, batched partial Cholesky with the
Schur contributions, level by level) followed by rsd_solve (FP64 PCG with the RSD
preconditioner to a relative residual of 1e-8, true residual re-checked in FP64).
Metric: DOF / (t_setup + t_solve) per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form mixed|fp64]
                  [--impl ours|reference] [--workload diffusion129|poisson13|...]

--impl reference times the CPU oracle (FP64, numpy/scipy on the host cores) on a bounded
sample of the same workload family.  Multi-GPU runs are independent replicas (the
single-problem workload is not sharded): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solve DOF/s to rel-res 1e-8, mixed vs FP64 form on 1 GB300; % of roofline"
TOL = 1e-8
# nominal dense tensor rates (PFLOP/s): used only to scale the measured BF16 peak to TF32
NOMINAL_BF16, NOMINAL_TF32 = 2.25, 1.1
NOMINAL_FP64_TFLOPS = 1.25       # GB300 FP64 (CUDA cores), for the ALU-bound FP64 form
CPU_SAMPLE = dict(n=41, depth=3)  # bounded oracle sample of the diffusion workload family


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """Sample SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if bus_id:
                cmd += ["-i", bus_id]
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        loaded = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _bus_id(torch):
    try:
        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


def recorded_traffic(kernel_class: str, key: str):
    """DRAM bytes (read + write) per launch of a kernel class, from the committed ncu
    summary of the default workload; None when there is none for the class or when the
    kernel source has changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "gemm_traffic_diffusion129_mixed.json")
    if kernel_class != "gemm_tcgen05" or not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("key") != key:
        return None
    src = os.path.join(ROOT, "paper_1210_6266_gb300", "csrc", "gemm_tc.cu")
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec.get("source_sha256_16"):
        return None
    return rec["dram_bytes_per_launch"]


def make_workload(name: str, n: int | None = None, depth: int | None = None):
    import synth
    w = dict(synth.WORKLOADS[name])
    if w["kind"] == "batched":
        if n is not None or depth is not None:
            raise SystemExit("--n/--depth apply to single-problem workloads only")
        return synth.batched_poisson(w["count"], w["size_seed"], w["f_seed0"]), w
    if w["kind"] not in ("poisson", "lognormal"):
        raise SystemExit(f"workload {name} is not built yet")
    if n is not None:
        w["n"] = n
    if depth is not None:
        w["depth"] = depth
    return synth.make(name, n=n, depth=depth), w


def cpu_baseline(steps: int = 1) -> dict:
    """The oracle as it stands (FP64 exact recursive Schur + PCG, numpy/scipy) on a bounded
    sample of the diffusion workload family, timed on this host's cores."""
    import synth
    from oracle import problem
    w = synth.diffusion_lognormal(CPU_SAMPLE["n"], CPU_SAMPLE["depth"], 2, 3)
    rates = []
    for _ in range(steps):
        r = problem.solve_timed(w, TOL)
        rates.append(r["n_dof"] / (r["t_setup"] + r["t_solve"]))
    cores = os.cpu_count()
    return {"value": statistics.median(rates), "unit": "DOF/s", "cores": cores, "kind": "oracle",
            "sample": f"diffusion lognormal n={CPU_SAMPLE['n']} (={r['n_dof']} DOF), depth "
                      f"{CPU_SAMPLE['depth']}, FP64 dense fronts via numpy/LAPACK, {r['iters']} PCG it, "
                      f"relres {r['relres']:.1e}"}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(1)
    t0 = time.perf_counter()
    cb = cpu_baseline(args.steps)
    dt = time.perf_counter() - t0
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "DOF/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"diffusion lognormal (sample n={CPU_SAMPLE['n']}, depth {CPU_SAMPLE['depth']})",
                       "form": "fp64 oracle", "tol": TOL},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--mode", default="exact", choices=["exact", "paper"])
    ap.add_argument("--workload", default="diffusion129")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--wave", type=int, default=64, help="problems per hierarchy (batched workload)")
    ap.add_argument("--n", type=int, default=None, help="grid side override (a scaled sample, e.g. for profiling)")
    ap.add_argument("--depth", type=int, default=None, help="octree depth override")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1210_6266_gb300 import (RSD, RSD_MODE_EXACT, RSD_MODE_PAPER, RSD_PREC_FP64, RSD_PREC_TF32,
                                       grid_problem, launch_count)
    from paper_1210_6266_gb300 import build as _build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()

    def barrier():
        if world > 1:
            dist.barrier()

    work, wdesc = make_workload(args.workload, args.n, args.depth)
    batched = wdesc["kind"] == "batched"
    if batched:
        probs = [grid_problem(w["n"], w["depth"], w["kappa"], w["f"]) for w in work]
        n_dof = sum(p["n_dof"] for p in probs)
        waves = [probs[i:i + args.wave] for i in range(0, len(probs), args.wave)]
    else:
        prob = grid_problem(work["n"], work["depth"], work["kappa"], work["f"])
        n_dof = prob["n_dof"]
    if args.form == "mixed":
        prec = dict(prec_leaf=RSD_PREC_TF32, prec_mid=RSD_PREC_TF32, prec_root=RSD_PREC_TF32)
        dtype = "tf32"
    else:
        prec = dict(prec_leaf=RSD_PREC_FP64, prec_mid=RSD_PREC_FP64, prec_root=RSD_PREC_FP64)
        dtype = "f64"
    mode = RSD_MODE_PAPER if args.mode == "paper" else RSD_MODE_EXACT
    stream = torch.cuda.current_stream()

    def merge_prof(a, b):
        if a is None:
            return b
        for k, v in b.items():
            if isinstance(v, dict) and "ms" in v:
                for f in ("launches", "ms", "flops", "bytes"):
                    a[k][f] += v[f]
            elif k in ("host_analysis_ms", "host_issue_ms"):
                a[k] += v
            elif k == "host_parts_ms":
                a[k] = {q: a[k][q] + v[q] for q in v}
        return a

    def step(profile=False):
        if not batched:
            h = RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                          profile=profile, mode=mode, **prec)
            u, st = h.solve(prob["b"], tol=TOL)
            prof = h.profile() if profile else None
            info = h.info()
            h.close()
            return st, prof, info
        stats, prof, info = None, None, None
        for wv in waves:
            h = RSD.setup_batched(wv, profile=profile, **prec)
            b = torch.cat([p["b"] for p in wv])
            u, st = h.solve(b, tol=TOL)
            prof = merge_prof(prof, h.profile()) if profile else None
            inf = h.info()
            info = inf if info is None else {k: (info[k] + inf[k] if k in ("factor_bytes", "setup_flops", "device_bytes") else info[k]) for k in info}
            if stats is None or st["relres"] > stats["relres"]:
                stats = st
            h.close()
        return stats, prof, info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    clocks = Clocks(_bus_id(torch))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = launch_count()
    torch.cuda.synchronize()
    barrier()
    ev0.record(stream)
    stats, profs = [], []
    for _ in range(args.steps):
        st, prof, info = step(profile=True)
        stats.append(st)
        profs.append(prof)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = (launch_count() - l0) // args.steps
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n_dof / (ms / 1e3)

    # end to end through the C ABI from pinned host buffers
    src = probs if batched else [prob]
    host = [{k: p[k].cpu().pin_memory() for k in ("rowptr", "col", "val", "dof_node", "b")} for p in src]
    u_host = torch.empty(n_dof, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for hp in host for t in hp.values())
    d2h = u_host.numel() * u_host.element_size()
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        off = 0
        groups = [list(range(i, min(i + args.wave, len(src)))) for i in range(0, len(src), args.wave)] if batched else [[0]]
        for g in groups:
            hp = [dict(host[i], parent=src[i]["parent"]) for i in g]
            if batched:
                h = RSD.setup_batched(hp, **prec)
            else:
                h = RSD.setup(hp[0]["rowptr"], hp[0]["col"], hp[0]["val"], hp[0]["dof_node"], hp[0]["parent"],
                              mode=mode, **prec)
            b = torch.cat([x["b"] for x in hp]).to("cuda", non_blocking=True)
            u, _ = h.solve(b, tol=TOL)
            u_host[off:off + u.numel()].copy_(u, non_blocking=True)
            off += u.numel()
            torch.cuda.synchronize()
            h.close()
    e2e_ms = (time.perf_counter() - t0) / max(e2e_steps, 1) * 1e3 if e2e_steps else float("nan")

    if rank != 0:
        return
    # roofline of the dominant kernel class (largest device time inside the timed region)
    agg = {}
    for p in profs:
        for k, v in p.items():
            if k in ("host_analysis_ms", "host_parts_ms", "host_issue_ms"):
                agg.setdefault(k, []).append(v)
                continue
            a = agg.setdefault(k, dict(launches=0, ms=0.0, flops=0.0, bytes=0.0))
            for f in ("launches", "ms", "flops", "bytes"):
                a[f] += v[f]
    classes = {k: v for k, v in agg.items() if k not in ("host_analysis_ms", "host_parts_ms", "host_issue_ms")}
    dom = max(classes, key=lambda k: classes[k]["ms"])
    d = classes[dom]
    pk, src = peaks()
    if dom == "gemm_tcgen05":
        peak = pk["bf16_tflops_sustained"] * NOMINAL_TF32 / NOMINAL_BF16
        roof = {"bound": "tensor", "achieved": d["flops"] / (d["ms"] / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s"}
        peak_note = f"TF32 = {src} BF16 sustained x {NOMINAL_TF32}/{NOMINAL_BF16} (nominal ratio)"
    elif dom in ("gemm_simt", "diag_factor", "panel_solve_simt") and args.form == "fp64":
        roof = {"bound": "alu", "achieved": d["flops"] / (d["ms"] / 1e3) / 1e12, "peak": NOMINAL_FP64_TFLOPS,
                "unit": "TFLOP/s"}
        peak_note = "FP64 CUDA-core nominal rate"
    else:
        roof = {"bound": "hbm", "achieved": d["bytes"] / (d["ms"] / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                "unit": "GB/s"}
        peak_note = f"{src} HBM copy bandwidth"
    roof["frac"] = roof["achieved"] / roof["peak"]
    wkey = f"{args.workload}/{args.form}/{args.mode}" if args.n is None and args.depth is None else "scaled"
    roof["traffic"] = recorded_traffic(dom, wkey)
    roof["kernel"] = dom
    roof["peak_source"] = peak_note
    roof["launches_per_step"] = d["launches"] / args.steps
    phase = {k: round(v["ms"] / args.steps, 3) for k, v in classes.items() if v["launches"]}
    sweeps = {k: classes[k] for k in ("sweep_up", "sweep_down")}
    sw_ms = sum(v["ms"] for v in sweeps.values())
    sw_gbs = sum(v["bytes"] for v in sweeps.values()) / (sw_ms / 1e3) / 1e9 if sw_ms else None
    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": (f"{args.workload}: -div(kappa grad u)=f, {work['n']}^3 nodes, trilinear hex, "
                                f"kappa lognormal per element") if wdesc["kind"] == "lognormal" else
                               (f"{args.workload}: {len(work)} independent Poisson problems, n in "
                                f"[{min(w['n'] for w in work)}, {max(w['n'] for w in work)}], 8-64 leaves each, "
                                f"hierarchies of {args.wave} problems") if batched else args.workload,
                   "n_dof": n_dof,
                   "subdomains": sum(8 ** w["depth"] for w in work) if batched else 8 ** work["depth"],
                   "merge_levels": max(w["depth"] for w in work) if batched else work["depth"],
                   "form": args.form, "mode": args.mode, "precisions": {k: v for k, v in prec.items()}, "tol": TOL,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (factors are tens of GB)"},
        "roofline": roof,
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": {"value": n_dof / (e2e_ms / 1e3), "unit": "DOF/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "detail": {"iterations": [s["iterations"] for s in stats], "relres": [s["relres"] for s in stats],
                   "ms_by_kernel_class": phase,
                   "host_analysis_ms": statistics.median(agg["host_analysis_ms"]),
                   "host_issue_ms": statistics.median(agg["host_issue_ms"]),
                   "host_parts_ms": agg["host_parts_ms"][-1],
                   "apply_sweeps_gbs": sw_gbs, "factor_bytes": info["factor_bytes"],
                   "setup_flops": info["setup_flops"], "device_bytes": info["device_bytes"]},
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(1)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
