"""Benchmark: solve throughput of the RSD-preconditioned FP64 PCG on one GB300.

One step = one pass of the whole path on resident inputs: rsd_setup (analysis of the
sub-domain tree and interface sets, front assembly, batched partial Cholesky with the
Schur contributions, level by level) followed by rsd_solve (FP64 PCG with the RSD
preconditioner to a relative residual of 1e-8, true residual re-checked in FP64).
Metric: DOF / (t_setup + t_solve) per step, mixed form against the plain FP64 form.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload diffusion129|...]
                  [--form mixed|fp64] [--mode exact|paper] [--gamma G] [--impl ours|reference]

The default run prints one JSON line: the mixed form (factor entries rounded to TF32, the
long Schur updates on FP16 operand copies, FP16 sweeps, FP64 PCG) on the 129^3 workload
(K timed steps after W warm-up steps) as the headline, and, in the same line, the plain
FP64 form of the same workload (one timed step: it takes over a minute), the 256-problem
batched workload in both forms (BF16 operands; the FP64 form on its first 64 problems),
paper mode with gamma = 8 inner GMRES iterations and FGMRES, the measured peaks of the
library's own GEMM kernels, and the oracle's CPU baseline.

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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solve DOF/s to rel-res 1e-8, mixed vs FP64 form on 1 GB300; % of roofline"
TOL = 1e-8
# nominal dense rates (the profiling recipe's table): used to scale the measured BF16 peak
# to TF32, and as the FP64 CUDA-core roof
NOMINAL_BF16, NOMINAL_TF32 = 2.25, 1.1
NOMINAL_FP64_TFLOPS = 1.25
CPU_SAMPLE = dict(n=41, depth=3)  # bounded oracle sample of the diffusion workload family
FP64_WARM = dict(n=33, depth=3)   # small grid that loads the FP64 kernels before the timed step
BATCH_FP64_SAMPLE = 64            # problems of the batched workload timed in the FP64 form
ELASTIC_NU = 0.3                  # Poisson's ratio of the elasticity workload


def job_rate(torch, dist, ms_local: float, units_per_rank: float, world: int, device: str):
    """Whole-job throughput of `world` replicas: all ranks' units over the slowest rank's
    time (the max over ranks of its ms per step).  Returns (units/s, ms)."""
    ms = ms_local
    if world > 1:
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * units_per_rank / (ms / 1e3), ms


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """Sample SM clocks and throttle reasons with nvidia-smi while the timed region runs
    (samples go to a temporary file that is removed afterwards)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.proc = None
        try:
            self.fh = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.path = self.fh.name
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if bus_id:
                cmd += ["-i", bus_id]
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
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        loaded = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "power_w_max": max(power) if power else None, "samples": len(sm)}


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
    if w["kind"] == "elasticity":
        if n is not None:
            w["n"] = n
        if depth is not None:
            w["depth"] = depth
        return dict(n=w["n"], depth=w["depth"], E_leaf=synth.elasticity_moduli(8 ** w["depth"], w["e_seed"]),
                    f=synth.uniform(w["f_seed"], 3 * (w["n"] - 2) ** 3)), w
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


PREC = None   # filled in main(): form name -> rsd_setup precision keywords


def prof_add(agg, p):
    """Sum rsd_profile dicts (kernel classes and host times)."""
    if p is None:
        return agg
    if agg is None:
        agg = {}
    for k, v in p.items():
        if isinstance(v, dict) and "ms" in v:
            a = agg.setdefault(k, dict(launches=0, ms=0.0, flops=0.0, bytes=0.0))
            for f in ("launches", "ms", "flops", "bytes"):
                a[f] += v[f]
        elif isinstance(v, dict):
            a = agg.setdefault(k, {})
            for q, x in v.items():
                a[q] = a.get(q, 0.0) + x
        else:
            agg[k] = agg.get(k, 0.0) + v
    return agg


def timed_steps(torch, run_one, steps: int):
    """Run `steps` steps; each returns (setup_done_event, stats, profile, info).  Returns
    ms per step (CUDA events on the current stream around all steps), the per-step setup
    and solve split, and the steps' results."""
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    marks = []
    ev0.record(stream)
    out = []
    for _ in range(steps):
        a = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        b, st, prof, info = run_one()
        c = torch.cuda.Event(enable_timing=True)
        c.record(stream)
        marks.append((a, b, c))
        out.append((st, prof, info))
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    su, so = [], []
    for (a, b, c), (st, _, _) in zip(marks, out):
        tot = a.elapsed_time(c)
        s = st["setup_ms_sum"] if "setup_ms_sum" in st else a.elapsed_time(b)
        su.append(s)
        so.append(tot - s)
    return ms, statistics.mean(su), statistics.mean(so), out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--mode", default="exact", choices=["exact", "paper"])
    ap.add_argument("--gamma", type=int, default=0, help="paper mode: inner GMRES iterations (0: dense S~)")
    ap.add_argument("--mixed-prec", default="fp16", choices=["tf32", "fp16", "bf16"],
                    help="factor precision of the mixed form (FP64 PCG in every form)")
    ap.add_argument("--workload", default="diffusion129")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-form record of the headline workload")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-workload record")
    ap.add_argument("--no-peaks", action="store_true", help="skip the GEMM peak probes")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper-mode (gamma = 8) record")
    ap.add_argument("--no-elastic", action="store_true", help="skip the elasticity-workload record")
    ap.add_argument("--tune", default="auto", choices=["auto", "off"],
                    help="auto: run the tile autotuner first and set up every hierarchy with its table")
    ap.add_argument("--wave", type=int, default=64, help="problems per hierarchy (batched workload)")
    ap.add_argument("--n", type=int, default=None, help="grid side override (a scaled sample, e.g. for profiling)")
    ap.add_argument("--depth", type=int, default=None, help="octree depth override")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    import paper_1210_6266_gb300 as rsd
    from paper_1210_6266_gb300 import build as _build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    global PREC
    mp = {"tf32": rsd.RSD_PREC_TF32, "fp16": rsd.RSD_PREC_FP16, "bf16": rsd.RSD_PREC_BF16}[args.mixed_prec]
    PREC = {"mixed": dict(prec_leaf=mp, prec_mid=mp, prec_root=mp),
            "fp64": dict(prec_leaf=rsd.RSD_PREC_FP64, prec_mid=rsd.RSD_PREC_FP64, prec_root=rsd.RSD_PREC_FP64)}
    DTYPE = {"mixed": {"tf32": "tf32", "fp16": "fp16+tf32", "bf16": "bf16+tf32"}[args.mixed_prec], "fp64": "f64"}
    mode = rsd.RSD_MODE_PAPER if args.mode == "paper" else rsd.RSD_MODE_EXACT
    single = world == 1
    pk, pk_src = peaks()

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- one step of a single problem / of a batch in waves ----------------------------
    tune_path, tune_rec = None, None
    if args.tune == "auto":
        tune_path = os.path.join(tempfile.mkdtemp(prefix="rsd_tune_"), "tune.json")
        secs = rsd.autotune(tune_path)
        tune_rec = {"seconds": secs, "buckets": rsd.tune_entries(tune_path),
                    "how": "rsd_autotune: tile width and split-K count of the tensor-core updates, per bucket of "
                           "output tiles x K and operand format, best of 3 synthetic launches each"}

    def single_step(prob, form, profile=False, m=mode, gamma=args.gamma):
        def run():
            h = rsd.RSD.setup(prob["rowptr"], prob["col"], prob["val"], prob["dof_node"], prob["parent"],
                              profile=profile, mode=m, gamma=gamma if m == rsd.RSD_MODE_PAPER else 0,
                              maxit=1000, tune_cache=tune_path, **PREC[form])
            b = torch.cuda.Event(enable_timing=True)
            b.record(torch.cuda.current_stream())
            u, st = h.solve(prob["b"], tol=TOL)
            prof = h.profile() if profile else None
            info = h.info()
            h.close()
            return b, st, prof, info
        return run

    def batched_step(waves, form, profile=False):
        # setup of every wave, then the solves: wave hierarchies are independent, so the
        # split is (all setups) + (all solves) per step; handles of earlier waves are closed
        # as soon as their solve is done, so the waves run one after another
        def run():
            stats, prof, info = None, None, None
            setup_ms = 0.0
            t_b = None
            for wv in waves:
                a = torch.cuda.Event(enable_timing=True)
                a.record(torch.cuda.current_stream())
                h = rsd.RSD.setup_batched(wv, profile=profile, tune_cache=tune_path, **PREC[form])
                t_b = torch.cuda.Event(enable_timing=True)
                t_b.record(torch.cuda.current_stream())
                t_b.synchronize()
                setup_ms += a.elapsed_time(t_b)
                b = torch.cat([p["b"] for p in wv])
                u, st = h.solve(b, tol=TOL)
                prof = prof_add(prof, h.profile()) if profile else None
                inf = h.info()
                info = inf if info is None else {k: (info[k] + inf[k] if k in ("factor_bytes", "setup_flops", "device_bytes", "n") else info[k]) for k in info}
                if stats is None:
                    stats = dict(st)
                else:
                    stats["relres"] = max(stats["relres"], st["relres"])
                    stats["iterations"] = max(stats["iterations"], st["iterations"])
                h.close()
            stats["setup_ms_sum"] = setup_ms
            return t_b, stats, prof, info
        return run

    # ---- peaks of the library's own GEMM kernels (roofline denominators) -------------
    peak_rec = None
    if single and not args.no_peaks:
        tf_b, tf_s = rsd.peak_gemm(rsd.RSD_PREC_TF32, 8192, reps=5, seconds=4.0)
        h_b, h_s = rsd.peak_gemm(rsd.RSD_PREC_FP16, 8192, reps=5, seconds=4.0)
        f64_b, f64_s = rsd.peak_gemm(rsd.RSD_PREC_FP64, 4096, reps=3, seconds=2.0)
        peak_rec = {"tf32_tcgen05": {"best": tf_b, "sustained": tf_s, "unit": "TFLOP/s",
                                     "how": "rsd_peak_gemm: the persistent 128x256 tcgen05 kind::tf32 kernel, "
                                            "C -= A B^T at 8192^3, best of 5 launches and back to back for 4 s"},
                    "fp16_tcgen05": {"best": h_b, "sustained": h_s, "unit": "TFLOP/s",
                                     "how": "rsd_peak_gemm: the same kernel with FP16 operands (kind::f16), "
                                            "8192^3, best of 5 launches and back to back for 4 s"},
                    "fp64_simt": {"best": f64_b, "sustained": f64_s, "unit": "TFLOP/s",
                                  "how": "rsd_peak_gemm: the FP64 CUDA-core 64x64-tile kernel, C -= A B^T at "
                                         "4096^3, best of 3 launches and back to back for 2 s"}}

    # ---- headline: the requested form on the requested workload ----------------------
    work, wdesc = make_workload(args.workload, args.n, args.depth)
    batched = wdesc["kind"] == "batched"
    if batched:
        probs = [rsd.grid_problem(w["n"], w["depth"], w["kappa"], w["f"]) for w in work]
        n_dof = sum(p["n_dof"] for p in probs)
        waves = [probs[i:i + args.wave] for i in range(0, len(probs), args.wave)]
        step = lambda form, profile=False: batched_step(waves, form, profile)  # noqa: E731
    elif wdesc["kind"] == "elasticity":
        prob = rsd.grid_problem_elastic(work["n"], work["depth"], work["E_leaf"], ELASTIC_NU, work["f"])
        n_dof = prob["n_dof"]
        step = lambda form, profile=False: single_step(prob, form, profile)  # noqa: E731
    else:
        prob = rsd.grid_problem(work["n"], work["depth"], work["kappa"], work["f"])
        n_dof = prob["n_dof"]
        step = lambda form, profile=False: single_step(prob, form, profile)  # noqa: E731

    for _ in range(args.warmup):
        step(args.form)()
    torch.cuda.synchronize()
    barrier()
    clocks = Clocks(_bus_id(torch))
    l0 = rsd.launch_count()
    barrier()
    ms, t_setup, t_solve, res = timed_steps(torch, step(args.form), args.steps)
    barrier()
    launches = (rsd.launch_count() - l0) // args.steps
    # the per-kernel breakdown and the roofline come from the same number of steps timed
    # again with CUDA events around every launch (a few per cent slower, not the headline)
    ms_prof, _, _, res_prof = timed_steps(torch, step(args.form, profile=True), args.steps)
    barrier()
    clk = clocks.stop()
    value, ms = job_rate(torch, dist, ms, n_dof, world, "cuda")
    stats = [r[0] for r in res]

    # ---- end to end through the C ABI from pinned host buffers ------------------------
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
                h = rsd.RSD.setup_batched(hp, tune_cache=tune_path, **PREC[args.form])
            else:
                h = rsd.RSD.setup(hp[0]["rowptr"], hp[0]["col"], hp[0]["val"], hp[0]["dof_node"], hp[0]["parent"],
                                  mode=mode, gamma=args.gamma if mode == rsd.RSD_MODE_PAPER else 0, maxit=1000,
                                  tune_cache=tune_path, **PREC[args.form])
            b = torch.cat([x["b"] for x in hp]).to("cuda", non_blocking=True)
            u, _ = h.solve(b, tol=TOL)
            u_host[off:off + u.numel()].copy_(u, non_blocking=True)
            off += u.numel()
            torch.cuda.synchronize()
            h.close()
    e2e_ms = (time.perf_counter() - t0) / max(e2e_steps, 1) * 1e3 if e2e_steps else float("nan")

    # ---- the FP64 form of the same workload and the batched workload (1 GPU only) ------
    fp64_rec, batch_rec = None, None
    headline_fp64_done = args.form == "fp64"
    if single and not args.no_fp64 and not batched and args.form == "mixed" and args.mode == "exact":
        import synth
        wsm = synth.diffusion_lognormal(FP64_WARM["n"], FP64_WARM["depth"], 2, 3)
        psm = rsd.grid_problem(wsm["n"], wsm["depth"], wsm["kappa"], wsm["f"])
        single_step(psm, "fp64")()                     # loads the FP64 kernels
        ms64, ts64, tv64, r64 = timed_steps(torch, single_step(prob, "fp64", profile=True), 1)
        fp64_rec = form_record(r64, ms64, ts64, tv64, n_dof, 1, pk, peak_rec, "fp64")
        fp64_rec["steps"] = 1
        fp64_rec["warmup"] = f"one step of the {FP64_WARM['n']}^3 grid (same kernels), not timed"
        headline_fp64_done = True
    if single and not args.no_batched and not batched and args.workload == "diffusion129" and args.mode == "exact":
        bwork, _ = make_workload("batched256")
        bprobs = [rsd.grid_problem(w["n"], w["depth"], w["kappa"], w["f"]) for w in bwork]
        bdof = sum(p["n_dof"] for p in bprobs)
        bwaves = [bprobs[i:i + args.wave] for i in range(0, len(bprobs), args.wave)]
        PREC["batched"] = dict(prec_leaf=rsd.RSD_PREC_BF16, prec_mid=rsd.RSD_PREC_BF16, prec_root=rsd.RSD_PREC_BF16)
        batched_step(bwaves, "batched")()              # warm-up
        msb, tsb, tvb, rb = timed_steps(torch, batched_step(bwaves, "batched"), 2)
        prof_b = timed_steps(torch, batched_step(bwaves, "batched", profile=True), 2)
        mixed_b = form_record(rb, msb, tsb, tvb, bdof, 2, pk, peak_rec, "mixed (BF16 operands)", prof=(prof_b[3], prof_b[0]))
        mixed_b["steps"] = 2
        mixed_b["warmup"] = 1
        sample = bwaves[0][:BATCH_FP64_SAMPLE]
        sdof = sum(p["n_dof"] for p in sample)
        msf, tsf, tvf, rf = timed_steps(torch, batched_step([sample], "fp64", profile=True), 1)
        fp64_b = form_record(rf, msf, tsf, tvf, sdof, 1, pk, peak_rec, "fp64")
        fp64_b["steps"] = 1
        fp64_b["sample"] = f"the first {len(sample)} problems ({sdof} DOF) as one hierarchy"
        sizes = [w["n"] for w in bwork]
        batch_rec = {"workload": f"batched256: {len(bwork)} independent Poisson problems, n in [{min(sizes)}, {max(sizes)}], "
                                 f"8-64 leaves each, hierarchies of {args.wave} problems",
                     "n_dof": bdof, "mixed": mixed_b, "fp64": fp64_b,
                     "mixed_over_fp64": mixed_b["value"] / fp64_b["value"]}

    elastic_rec = None
    if single and not args.no_elastic and args.workload == "diffusion129" and args.mode == "exact" and args.form == "mixed":
        ework, _ = make_workload("elasticity97")
        eprob = rsd.grid_problem_elastic(ework["n"], ework["depth"], ework["E_leaf"], ELASTIC_NU, ework["f"])
        single_step(eprob, "mixed")()                 # warm-up
        mse, tse, tve, re_ = timed_steps(torch, single_step(eprob, "mixed"), 2)
        prof_e = timed_steps(torch, single_step(eprob, "mixed", profile=True), 2)
        elastic_rec = form_record(re_, mse, tse, tve, eprob["n_dof"], 2, pk, peak_rec, "mixed", prof=(prof_e[3], prof_e[0]))
        elastic_rec.update(workload=(f"elasticity97: 3-D linear elasticity (3 DOF/node), {ework['n']}^3 nodes, "
                                     f"trilinear hex, E per leaf log-uniform [1, 1e3], nu = {ELASTIC_NU}, "
                                     f"{8 ** ework['depth']} leaves (depth {ework['depth']})"),
                           n_dof=eprob["n_dof"], steps=2, warmup=1,
                           fp64_form="not timed: about 3.5e14 flops of FP64 factorisation, some 5 minutes")
        del eprob
    paper_rec = None
    if single and not args.no_paper and not batched and args.mode == "exact" and args.form == "mixed":
        single_step(prob, "mixed", m=rsd.RSD_MODE_PAPER, gamma=8)()          # warm-up
        msp, tsp, tvp, rp = timed_steps(torch, single_step(prob, "mixed", m=rsd.RSD_MODE_PAPER, gamma=8), 1)
        prof_p = timed_steps(torch, single_step(prob, "mixed", profile=True, m=rsd.RSD_MODE_PAPER, gamma=8), 1)
        paper_rec = form_record(rp, msp, tsp, tvp, n_dof, 1, pk, peak_rec, "mixed", prof=(prof_p[3], prof_p[0]))
        paper_rec.update(mode="paper (Algorithm 2, V-hat truncation)", gamma=8, krylov="FGMRES(30)", steps=1, warmup=1)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    head = form_record(res, ms, t_setup, t_solve, n_dof, args.steps, pk, peak_rec, args.form, prof=(res_prof, ms_prof))
    roof = head.pop("roofline")
    wkey = f"{args.workload}/{args.form}/{args.mode}" if args.n is None and args.depth is None else "scaled"
    roof["traffic"] = recorded_traffic(roof.get("kernel"), wkey)
    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.form], "data": "synthetic",
        "config": {"workload": (f"{args.workload}: -div(kappa grad u)=f, {work['n']}^3 nodes, trilinear hex, "
                                f"kappa lognormal per element") if wdesc["kind"] == "lognormal" else
                               (f"{args.workload}: 3-D linear elasticity, {work['n']}^3 nodes, 3 DOF/node, E per leaf "
                                f"log-uniform [1, 1e3], nu = {ELASTIC_NU}") if wdesc["kind"] == "elasticity" else
                               (f"{args.workload}: {len(work)} independent Poisson problems, n in "
                                f"[{min(w['n'] for w in work)}, {max(w['n'] for w in work)}], 8-64 leaves each, "
                                f"hierarchies of {args.wave} problems") if batched else args.workload,
                   "n_dof": n_dof,
                   "subdomains": sum(8 ** w["depth"] for w in work) if batched else 8 ** work["depth"],
                   "merge_levels": max(w["depth"] for w in work) if batched else work["depth"],
                   "form": args.form, "mode": args.mode, "gamma": args.gamma if args.mode == "paper" else None,
                   "krylov": "FGMRES(30)" if args.mode == "paper" and args.gamma > 0 else "PCG",
                   "precisions": PREC[args.form], "tol": TOL,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (factors are tens of GB)"},
        "roofline": roof,
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": {"value": n_dof / (e2e_ms / 1e3), "unit": "DOF/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "setup_solve": {k: head[k] for k in ("t_setup_ms", "t_solve_ms", "setup_dof_s", "solve_dof_s")},
        "apply_roofline": head.pop("apply_roofline"),
        "detail": dict(head.pop("detail"), iterations=[s["iterations"] for s in stats],
                       relres=[s["relres"] for s in stats]),
    }
    if fp64_rec is not None:
        line["fp64_form"] = fp64_rec
        line["mixed_over_fp64"] = value / fp64_rec["value"]
    if batch_rec is not None:
        line["batched256"] = batch_rec
    if paper_rec is not None:
        line["paper_gamma8"] = paper_rec
    if elastic_rec is not None:
        line["elasticity97"] = elastic_rec
    if peak_rec is not None:
        line["peaks_measured"] = peak_rec
    line["autotune"] = tune_rec
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(1)
    print(json.dumps(line), flush=True)
    rsd._lib.load().rsd_release_cache()
    if world > 1:
        dist.destroy_process_group()


def form_record(res, ms, t_setup, t_solve, n_dof, steps, pk, peak_rec, form, prof=None) -> dict:
    """Throughput, setup/solve split and rooflines of one form's timed steps.  prof = (results,
    ms per step) of the same steps timed again with per-launch events: the kernel classes
    come from there when given, else from `res` (which then carries the events itself)."""
    stats = [r[0] for r in res]
    agg = None
    for r in (prof[0] if prof is not None else res):
        agg = prof_add(agg, r[1])
    info = res[-1][2]
    classes = {k: v for k, v in agg.items() if isinstance(v, dict) and "ms" in v}
    per = {k: v["ms"] / steps for k, v in classes.items() if v["launches"]}
    # setup: the tensor-core (or CUDA-core) GEMM classes against the algorithmic flops
    # sum_t (s^3/3 + s^2 b + s b^2), shared between the classes in proportion to their
    # counted flops; each class has the peak of its own operand type, and the roof of the
    # whole is the sum of the classes' times at their peaks
    tc_classes = [k for k in ("gemm_tcgen05_f16", "gemm_tcgen05") if classes.get(k, {}).get("launches")]
    if tc_classes:
        bf = pk["bf16_tflops_sustained"]
        cls_peak = {"gemm_tcgen05": bf * NOMINAL_TF32 / NOMINAL_BF16, "gemm_tcgen05_f16": bf}
        counted = sum(classes[k]["flops"] for k in tc_classes)
        per_cls, t_min, t_act = {}, 0.0, 0.0
        for k in tc_classes:
            fl = info["setup_flops"] * classes[k]["flops"] / counted
            ms_k = classes[k]["ms"] / steps
            per_cls[k] = {"algorithmic_flops": fl, "ms": ms_k, "achieved": fl / (ms_k / 1e3) / 1e12,
                          "peak": cls_peak[k], "frac": fl / (ms_k / 1e3) / 1e12 / cls_peak[k],
                          "launches": classes[k]["launches"] / steps}
            t_min += fl / (cls_peak[k] * 1e12)
            t_act += ms_k / 1e3
        achieved = info["setup_flops"] / t_act / 1e12
        peak = info["setup_flops"] / t_min / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_source": (f"measured BF16 sustained {bf} TFLOP/s for the kind::f16 launches (FP16 and BF16 "
                                f"share the dense rate), x {NOMINAL_TF32}/{NOMINAL_BF16} (nominal ratio) for the "
                                f"kind::tf32 launches; the peak is the flop-weighted combination"),
                "classes": per_cls}
        if peak_rec:
            own = {"gemm_tcgen05": peak_rec["tf32_tcgen05"]["sustained"],
                   "gemm_tcgen05_f16": peak_rec["fp16_tcgen05"]["sustained"]}
            t_own = sum(per_cls[k]["algorithmic_flops"] / (own[k] * 1e12) for k in tc_classes)
            roof["frac_of_own_kernel_peak"] = t_own / t_act
        gemm_cls = "+".join(tc_classes)
        g_launches = sum(classes[k]["launches"] for k in tc_classes)
    else:
        g = classes["gemm_simt"]
        g_ms = g["ms"] / steps
        achieved = info["setup_flops"] / (g_ms / 1e3) / 1e12 if g_ms else None
        roof = {"bound": "alu", "achieved": achieved, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                "peak_source": "FP64 CUDA-core nominal rate (152 SMs at 2.07 GHz)"}
        if peak_rec:
            roof["fp64_measured_sustained"] = peak_rec["fp64_simt"]["sustained"]
            roof["frac_of_fp64_measured"] = achieved / peak_rec["fp64_simt"]["sustained"]
        gemm_cls = "gemm_simt"
        g_launches = g["launches"]
    roof["frac"] = achieved / roof["peak"] if achieved else None
    roof["kernel"] = gemm_cls
    roof["achieved_basis"] = "rsd_info setup_flops = sum_t (s^3/3 + s^2 b + s b^2) / the classes' summed launch time"
    roof["launches_per_step"] = g_launches / steps
    sw = [classes.get(k) for k in ("sweep_up", "sweep_down") if classes.get(k)]
    sw_ms = sum(v["ms"] for v in sw) / steps
    sw_bytes = sum(v["bytes"] for v in sw) / steps
    apply_roof = None
    if sw_ms:
        apply_roof = {"bound": "hbm", "achieved": sw_bytes / (sw_ms / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                      "unit": "GB/s", "kernel": "k_fwd_sweep + k_bwd_sweep",
                      "bytes_per_step": sw_bytes, "ms_per_step": sw_ms,
                      "applications_per_step": statistics.mean(s["iterations"] for s in stats)}
        apply_roof["frac"] = apply_roof["achieved"] / apply_roof["peak"]
    smv = classes.get("gamma_smv")
    smv_roof = None
    if smv and smv["ms"]:
        # paper mode, gamma > 0: the S-MatVecs' leaf-coupling products stream the X rows
        # of the leaves that couple to the interface level twice (X^T x, then X t)
        smv_roof = {"bound": "hbm", "achieved": smv["bytes"] / (smv["ms"] / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                    "unit": "GB/s", "kernel": "k_smv_leaf + k_smv_rows", "bytes_per_step": smv["bytes"] / steps,
                    "ms_per_step": smv["ms"] / steps, "launches_per_step": smv["launches"] / steps}
        smv_roof["frac"] = smv_roof["achieved"] / smv_roof["peak"]
    return {
        "value": n_dof / (ms / 1e3), "unit": "DOF/s", "ms_per_step": ms, "form": form,
        "t_setup_ms": t_setup, "t_solve_ms": t_solve,
        "setup_dof_s": n_dof / (t_setup / 1e3), "solve_dof_s": n_dof / (t_solve / 1e3),
        "iterations": [s["iterations"] for s in stats], "relres": [s["relres"] for s in stats],
        "roofline": roof, "apply_roofline": apply_roof, **({"smv_roofline": smv_roof} if smv_roof else {}),
        "detail": {"ms_by_kernel_class": {k: round(v, 3) for k, v in per.items()},
                   "ms_per_step_with_launch_events": prof[1] if prof is not None else ms,
                   "host_analysis_ms": agg.get("host_analysis_ms", 0.0) / steps,
                   "host_issue_ms": agg.get("host_issue_ms", 0.0) / steps,
                   "factor_bytes": info["factor_bytes"], "setup_flops": info["setup_flops"],
                   "device_bytes": info["device_bytes"]},
    }


if __name__ == "__main__":
    main()
