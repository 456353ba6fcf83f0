"""Benchmark of the per-level implicit diffusion solve on one GB300 (or N replicas).

Default workload (one "step" = every row of the hot path over one batch):
  512 independent single-level backward-Euler solves of ragged sizes (oct
  counts log-uniform over 8^3..64^3 cells, near-cubic oct boxes), per-solve dt
  log-uniform over 1e-3..1e2 x the explicit CFL step, K log-normal (sigma 1)
  per cell, random Dirichlet / zero-flux walls; per step: build every level
  operator and right-hand side on the device, then solve all 512 in one
  batched, graph-replayed launch sequence in mixed precision (FP32 bulk, FP64
  dots) with FP64 iterative refinement until the FP64 certificate
  ||b - A x|| <= 5e-11 ||x|| holds (the level matrix has lambda_min >= 1, so
  the result is within 5e-11 of the exact solution and within 1e-10 of the
  oracle's, which stops on the same rule).

Metric: level-solves/s (whole job), with the dominant kernel's achieved HBM
bandwidth against the measured peak, the plain per-solve FP64 GPU path on the
same mix, and the FP64 CPU oracle on a bounded sample (one thread and every
host core), with the error of each GPU path against it.

Other legs on the same line (each can be switched off): the end-to-end
number through pinned host buffers (inputs of the next step copied during
the solve); the same batch with Crank-Nicolson steps; the served request
stream (p50 / p99 latency against plain FP64 one at a time); the two-level
AMR step with each interface row; the paper's equilibrium test (uniform and
adaptive) and its Dirac test with a mesh that follows the gradient criterion.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

For N > 1 it runs under torch.distributed.run; each rank solves its own
512-solve batch (a different seed): independent problems, no data-path
collective, weak scaling.
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

import workloads as W  # noqa: E402

METRIC = "stencil-PCG GB/s vs HBM peak; level-solves/s and p50/p99 latency vs plain FP64"
UNIT = "level-solves/s"
TOL = 5e-11  # certified: ||b - A x|| <= TOL ||x||, so the relative error is <= TOL


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(rank: int) -> int:
    """Each rank solves its own batch of independent solves (weak scaling):
    the workload seed of rank r."""
    return 1404 + 1000 * rank


def reduce_max(value: float, device=None) -> float:
    """Max over ranks of a per-rank time (no-op without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms during the
    timed region: sampling starts (and its first sample is awaited) before
    the region, each line is stamped on arrival, and only the lines that
    arrived inside the region are summarised (all lines if none did, which
    "samples_in_region": 0 then says)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, gpu_id: str):
        # nvidia-smi numbers GPUs physically and ignores CUDA_VISIBLE_DEVICES,
        # so the sampler is given a stable identifier of the GPU in use (its
        # UUID, else its PCI bus id; see smi_gpu_id), never a CUDA ordinal
        self.gpu = str(gpu_id)
        self.proc = None
        self.lines = []  # (arrival time, line)
        self._t = None
        self._first = threading.Event()

    def start(self, wait_s: float = 3.0):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        self._first.wait(wait_s)  # sampling is live before the caller's region starts

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))
            self._first.set()

    def stop(self, t0=None, t1=None):
        """Summary of the samples that arrived in [t0, t1 + one period]
        (perf_counter times; None: every sample)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "gpu": self.gpu}
        time.sleep(2.0 * self.PERIOD_MS / 1e3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        lines = list(self.lines)
        inside = lines
        if t0 is not None and t1 is not None:
            inside = [(t, ln) for t, ln in lines if t0 <= t <= t1 + self.PERIOD_MS / 1e3]
        summary = self._summarise(inside if inside else lines)
        summary["gpu"] = self.gpu
        summary["samples_in_region"] = len(inside) if (t0 is not None and t1 is not None) else summary["samples"]
        return summary

    @staticmethod
    def _summarise(lines):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons),
            "samples": len(sm),
        }


def smi_gpu_id(local: int) -> str:
    """nvidia-smi's identifier of CUDA device `local` of this process: its
    UUID ("GPU-..."), else its PCI bus id, else (neither known) the ordinal
    itself, which is only right when no CUDA_VISIBLE_DEVICES remapping is in
    force."""
    import torch

    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    try:
        p = torch.cuda.get_device_properties(local)
        return "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        pass
    return str(local)


def _traffic_for(kernel: str, alg_bytes_per_launch: float):
    """DRAM bytes per launch of a kernel, from the committed ncu capture
    (profiles/ncu_traffic.json) when it was taken on the current kernel
    source: the captured launch's DRAM / algorithmic byte ratio applied to
    this run's average launch.  None otherwise."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        import hashlib

        d = json.load(open(p))
        src = open(os.path.join(ROOT, "paper_1401_1112_gb300", "csrc", "kernels.cu"), "rb").read()
        if d.get("kernels_cu_sha256") != hashlib.sha256(src).hexdigest():
            return None
        k = d["kernels"].get(kernel)
        if not k:
            return None
        return round(k["dram_bytes"] / k["algorithmic_bytes"] * alg_bytes_per_launch)
    except (OSError, ValueError, KeyError):
        return None


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local):
    import torch

    from paper_1401_1112_gb300 import ats, build

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # one non-default stream for torch's work and the library's, so that the
    # per-step copies and the solves are ordered (and graphs can be captured)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    solves = W.ragged_batch(n_solves=args.solves, seed=replica_seed(rank))
    n = len(solves)
    sizes = [lv.n_cell for lv, _ in solves]
    total_cells = int(sum(sizes))
    offs = np.concatenate([[0], np.cumsum(sizes)])
    fsz = [lv.n_face for lv, _ in solves]
    foffs = np.concatenate([[0], np.cumsum(fsz)])

    # device-resident inputs (flat, with per-solve views)
    K_h = np.concatenate([st.K for _, st in solves])
    E_h = np.concatenate([st.E for _, st in solves])
    fE_h = np.concatenate([st.face_E for _, st in solves]) if foffs[-1] else np.zeros(1)
    fF_h = np.concatenate([st.face_F for _, st in solves]) if foffs[-1] else np.zeros(1)
    K_d = torch.from_numpy(K_h).to(dev)
    E_d = torch.from_numpy(E_h).to(dev)
    fE_d = torch.from_numpy(fE_h).to(dev)
    fF_d = torch.from_numpy(fF_h).to(dev)
    x_d = torch.empty_like(E_d)

    ctx = ats.Context(local)
    ctx.set_stream(stream.cuda_stream)
    t0 = time.time()
    levels = [ats.Level(ctx, lv) for lv, _ in solves]
    layout_s = time.time() - t0

    def view(t, a, b):
        return t[int(a):int(b)]

    def coef_kwargs(k):
        st = solves[k][1]
        fa, fb = foffs[k], foffs[k + 1]
        has_f = fb > fa
        return dict(dt=st.dt, K=view(K_d, offs[k], offs[k + 1]), E_old=view(E_d, offs[k], offs[k + 1]),
                    face_E=view(fE_d, fa, fb) if has_f else None, face_F=view(fF_d, fa, fb) if has_f else None)

    xs = [view(x_d, offs[k], offs[k + 1]) for k in range(n)]
    for k in range(n):  # per-level entry point once (the plan needs built operators)
        levels[k].build(**coef_kwargs(k))
    # every level of the batch on the resident solver (levels up to
    # --res-max-octs octs; the batch's largest has 32 768)
    batch = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                      use_graph=1, check_every=args.check_every, mem=ats.ATS_MEM_DEVICE, tile_octs=args.tile,
                      inner_rtol=args.inner_rtol, res_max_octs=args.res_max_octs, cg_form=args.cg_form)
    coefs = batch.prepare_coefs([coef_kwargs(k) for k in range(n)])

    def build_ops():
        batch.build_operators(coefs)  # all levels' coefficients and right-hand sides, one launch

    # work-item size and poll interval chosen by the library's autotuner on
    # these solves (before the warm-up; not timed)
    tune = None
    if not args.no_autotune and args.tile == 0:
        build_ops()
        x_d.copy_(E_d)
        t_tune = time.time()
        tune = batch.autotune(xs, reps=2)
        tune["seconds"] = round(time.time() - t_tune, 2)
    tile_octs = tune["tile_octs"] if tune else args.tile
    check_every = tune["check_every"] if tune else args.check_every
    # the resident shape of the tuned plan, for the other batches of this run
    res_shape = dict(res_max_octs=args.res_max_octs, cg_form=args.cg_form)
    if tune:
        res_shape.update(res_threads=tune["chosen"]["res_threads"], res_cluster=tune["chosen"]["res_cluster"],
                         res_cta_octs=tune["chosen"]["res_cta_octs"])
        tune.pop("chosen")

    def step():
        x_d.copy_(E_d)          # initial guess x0 = E^n
        build_ops()             # coefficients, interface terms, right-hand side
        code, stats = batch.solve(xs)
        if code < 0:  # a warning (ATS_WARN_NEGATIVE) is a result
            raise RuntimeError(f"batch solve failed: {code} {ats.ats_last_error()}")
        return stats

    for _ in range(args.warmup):
        stats = step()
    torch.cuda.synchronize()

    dist = None
    if world > 1:
        import torch.distributed as dist

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    batch.set_profiling(True)
    sampler = ClockSampler(smi_gpu_id(local))
    sampler.start()
    barrier()
    t_region = time.perf_counter()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    acc = {"op_ms": 0.0, "op_bytes": 0.0, "ref_ms": 0.0, "ref_bytes": 0.0, "upd_ms": 0.0, "upd_bytes": 0.0,
           "ticks": 0, "res_ms": 0.0, "res_bytes": 0.0, "res_launches": 0}
    res_timeline = []
    launches = 0
    ev0.record(stream)
    for _ in range(args.steps):
        stats = step()
        ks = batch.kernel_stats()
        for key in acc:
            acc[key] += ks[key]
        res_timeline.append({k: ks[k] for k in ("res_span_ms", "res_longest_ms", "res_occupancy", "res_longest",
                                                "res_grid", "res_solves")})
        # tick kernels, resident launches, operator build (2), init, final, flag gather
        launches += ks["launches"] + ks["res_launches"] + 5
    ev1.record(stream)
    barrier()
    clocks = sampler.stop(t_region, time.perf_counter())
    ms = reduce_max(ev0.elapsed_time(ev1), dev)
    batch.set_profiling(False)
    value = n * args.steps * world / (ms / 1e3)
    iters = [s["iterations"] for s in stats]
    cell_its = int(sum(int(s["iterations"]) * int(sz) for s, sz in zip(stats, sizes)))  # per step
    refs = [s["refinements"] for s in stats]
    bounds = [s["err_bound"] for s in stats]

    # dominant kernel roofline (algorithmic bytes / event-timed duration).
    # k_ref (the FP64 residual, bound by the FP64 ALU) runs on a second stream
    # concurrently with k_op, so its event span includes time shared with k_op:
    # the roofline kernel is the longer of the two HBM-bound CG kernels.
    peak, peak_kind = _peaks()
    # the resident launch (a cluster kernel and, beside it, single CTAs on the
    # SMs no cluster fits on) counts as one launch per step: its span
    res_name = "k_res2_cluster+k_res2_cta"
    kern = {"k_op<float>": ("op_ms", "op_bytes"), "k_ref<float>": ("ref_ms", "ref_bytes"),
            "k_upd<float>": ("upd_ms", "upd_bytes"), res_name: ("res_ms", "res_bytes")}
    dom = max(("k_op<float>", "k_upd<float>", res_name), key=lambda k: acc[kern[k][0]])
    dms, dbytes = acc[kern[dom][0]], acc[kern[dom][1]]
    dl = args.steps if dom == res_name else max(1, acc["ticks"])
    achieved = dbytes / (dms / 1e3) / 1e9 if dms > 0 else 0.0
    roofline = {
        "bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
        "frac": round(achieved / peak, 4), "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
        "traffic": _traffic_for(dom, dbytes / dl),
        "launches": int(dl), "bytes_per_launch": round(dbytes / dl),
        # the whole step on the minimal Jacobi-PCG traffic: 10 words per cell
        # and CG iteration (read p, K, x, r, q, D^-1; write q, x, r, p)
        "cg_step": {"cell_iterations": cell_its, "bytes_per_cell_iteration": 10 * 4,
                    "achieved": round(cell_its * 40.0 / (ms / args.steps / 1e3) / 1e9, 1),
                    "frac": round(cell_its * 40.0 / (ms / args.steps / 1e3) / 1e9 / peak, 4)},
        "per_kernel": {k: {"ms": round(acc[a], 3),
                           "GBps": round(acc[b] / (acc[a] / 1e3) / 1e9, 1) if acc[a] else None,
                           "bound": "fp64 alu, concurrent with k_op" if k.startswith("k_ref") else "hbm"}
                       for k, (a, b) in kern.items()},
        "resident_timeline": res_timeline[-1] if res_timeline else None,
    }

    # end to end through the public API with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        Kp = torch.from_numpy(K_h).pin_memory()
        Ep = torch.from_numpy(E_h).pin_memory()
        fEp = torch.from_numpy(fE_h).pin_memory()
        fFp = torch.from_numpy(fF_h).pin_memory()
        xp = torch.empty_like(Ep).pin_memory()
        Kn, En, fEn, fFn, xn = Kp.numpy(), Ep.numpy(), fEp.numpy(), fFp.numpy(), xp.numpy()
        # x0 = E^n of the build (the paper's initial guess): x is output only
        # the whole tick loop as one graph (device-side WHILE node): the host
        # waits once per solve
        hbatch = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                           use_graph=2, check_every=check_every, tile_octs=tile_octs, mem=ats.ATS_MEM_HOST,
                           x0=ats.ATS_X0_E_OLD, **res_shape)
        hx = [xn[offs[k]:offs[k + 1]] for k in range(n)]

        hcoefs = hbatch.prepare_coefs([
            dict(dt=solves[k][1].dt, K=Kn[offs[k]:offs[k + 1]], E_old=En[offs[k]:offs[k + 1]],
                 face_E=fEn[foffs[k]:foffs[k + 1]] if foffs[k + 1] > foffs[k] else None,
                 face_F=fFn[foffs[k]:foffs[k + 1]] if foffs[k + 1] > foffs[k] else None) for k in range(n)])

        # each step: its inputs from pinned host memory (copied on the batch's
        # copy stream while the previous step's solve runs, then built), the
        # solve, the solution back to pinned host memory
        def e2e_step():
            hbatch.build_operators(hcoefs)   # this step's operators, from the prefetched copies
            hbatch.prefetch_operators(hcoefs)  # the next step's inputs, overlapping this solve
            code, _ = hbatch.solve(hx)
            if code < 0:  # a warning (ATS_WARN_NEGATIVE) is a result
                raise RuntimeError("e2e solve failed")

        hbatch.prefetch_operators(hcoefs)
        e2e_step()
        barrier()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        e_s = reduce_max(time.perf_counter() - t1, dev)
        h2d = int(K_h.nbytes + E_h.nbytes + (fE_h.nbytes + fF_h.nbytes if foffs[-1] else 0))
        e2e = {"value": round(n * args.steps * world / e_s, 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(E_h.nbytes)}
        hbatch.close()

    # the last timed step's solutions (mixed, refined), for the error vs the oracle
    results = {}
    if rank == 0 and not args.no_cpu:
        xh = x_d.cpu().numpy()
        results["mixed_refined"] = [xh[offs[k]:offs[k + 1]].copy() for k in range(n)]

    # plain per-solve FP64 GPU path on the same mix (no batching, no graph)
    fp64 = None
    if not args.no_fp64 and rank == 0:
        build_ops()
        x_d.copy_(E_d)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for k in range(n):
            code, _ = ats.ats_solve(levels[k].handle, xs[k], opts=ats.make_opts(
                tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_FP64,
                check_every=args.check_every, mem=ats.ATS_MEM_DEVICE))
            if code < 0:  # a warning (ATS_WARN_NEGATIVE) is a result
                raise RuntimeError("fp64 solve failed")
        torch.cuda.synchronize()
        f_s = time.perf_counter() - t1
        fp64 = {"value": round(n / f_s, 2), "unit": UNIT, "path": "plain per-solve FP64 PCG, one solve at a time"}
        if not args.no_cpu:
            xh = x_d.cpu().numpy()
            results["fp64"] = [xh[offs[k]:offs[k + 1]].copy() for k in range(n)]

    # the mixed path without FP64 refinement: one FP32 inner solve from the
    # FP64 residual of x0 = E^n, to a 1e-6 reduction (the FP32 floor); the
    # final true-residual pass only measures it (status NOT_CONVERGED)
    if rank == 0 and not args.no_cpu:
        ubatch = ats.Batch(ctx, levels, tol=TOL, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED,
                           use_graph=1, check_every=check_every, tile_octs=tile_octs, mem=ats.ATS_MEM_DEVICE,
                           max_refine=1, inner_rtol=1e-6, **res_shape)
        build_ops()
        x_d.copy_(E_d)
        code, _ = ubatch.solve(xs)
        if code < 0 and code != ats.ATS_ERR_NOT_CONVERGED:
            raise RuntimeError(f"unrefined batch failed: {code}")
        ubatch.close()
        xh = x_d.cpu().numpy()
        results["mixed_unrefined"] = [xh[offs[k]:offs[k + 1]].copy() for k in range(n)]

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(solves, budget_s=args.cpu_seconds, gpu_results=results)

    serve = None
    if rank == 0 and not args.no_serve:
        serve = run_serve(args, ats, local)
        if e2e is not None:
            # the served stream is measured end to end through the public
            # serving calls (submit / wait, host arrays): its latencies travel
            # with the end-to-end figure
            e2e["served"] = {k: serve[k] for k in ("requests", "of", "throughput", "p50_ms", "p99_ms",
                                                   "arrival_rate_per_s")}
            e2e["served"]["fp64_per_solve"] = {k: serve["fp64_per_solve"][k]
                                               for k in ("throughput", "p50_ms", "p99_ms")}
            e2e["served"]["oracle_check_ok"] = all(c["within_bound"] for c in serve["oracle_check"])

    amr = None
    if rank == 0 and not args.no_amr:
        amr = run_amr_interfaces(ats, ctx)

    fld_amr = None
    if rank == 0 and not args.no_fld:
        fld_amr = run_fld_amr(ats, ctx)
    equilibrium = None
    if rank == 0 and not args.no_equilibrium:
        equilibrium = run_equilibrium(ats, ctx)
    dirac = None
    if rank == 0 and not args.no_dirac:
        dirac = run_dirac(ats, ctx)

    # the same batch integrated with Crank-Nicolson (half-step backward-Euler
    # operator, E^{n+1} = 2 x' - E^n in the copy-out), device-resident inputs
    cn = None
    if rank == 0 and not args.no_cn:
        cn_coefs = batch.prepare_coefs([dict(coef_kwargs(k), integrator=ats.ATS_INTEGRATOR_CRANK_NICOLSON)
                                        for k in range(n)])

        def cn_step():
            x_d.copy_(E_d)
            batch.build_operators(cn_coefs)
            code, st = batch.solve(xs)
            if code < 0:  # a warning (ATS_WARN_NEGATIVE) is a result
                raise RuntimeError(f"Crank-Nicolson batch failed: {code}")
            return st

        cn_step()
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.steps):
            cst = cn_step()
        c1.record(stream)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1) / args.steps
        cn = {"value": round(n / (cms / 1e3), 2), "unit": UNIT, "ms_per_step": round(cms, 3),
              "iterations_mean": float(np.mean([s["iterations"] for s in cst])),
              "iterations_max": int(np.max([s["iterations"] for s in cst])),
              "workload": "the same batch, one Crank-Nicolson step per solve"}

    batch.close()
    for L in levels:
        L.close()
    ctx.close()
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {
            "workload": f"batched level solves: {n} ragged single-level backward-Euler solves, 8^3..64^3 cells, "
                        f"mixed FP32/FP64 PCG + FP64 refinement to the certificate ||b - Ax|| <= 5e-11 ||x||, "
                        f"graph-replayed",
            "solves": n, "cells": total_cells, "tol": TOL, "seed": 1404,
            "l2": "inputs larger than L2 (working set ~%.2f GB)" % (total_cells * 64 / 1e9),
            "parallelism": f"replicas x{world}",
            "tile_octs": tile_octs, "check_every": check_every, "autotune": tune,
            "scheduler": "resident solver for levels up to %d octs (one launch runs every solve to its end: "
                         "thread-block clusters, CG state in shared memory)" % args.res_max_octs,
        },
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "fp64_per_solve": fp64,
        "serve": serve,
        "amr_interfaces": amr,
        "crank_nicolson": cn,
        "equilibrium_1d": equilibrium,
        "fld_amr": fld_amr,
        "dirac_1d": dirac,
        "solve_stats": {"iterations_mean": float(np.mean(iters)), "iterations_max": int(np.max(iters)),
                        "refinements_mean": float(np.mean(refs)),
                        "max_err_bound": float(np.max(bounds)), "layout_s": round(layout_s, 3)},
    }


def run_amr_interfaces(ats, ctx, coarse_steps=3, check_every=16):
    """The two-level workload (base 64^3, level 1 on the central 1/8 of the
    volume, Gaussian pulse, constant K, fine first) with each row of the
    coarse-to-fine faces: time per coarse step (two fine solves and one
    coarse solve, mixed precision, certified 5e-11) as one captured graph
    (use_graph = 3) and with deferred solves (use_graph = 2), and the
    relative change of the total energy per step (zero-flux walls: only the
    interfaces can change it; the Neumann rows with the stored flux conserve
    it)."""
    levels, states, dt = W.two_level_gaussian_64cube(n0=64)

    def energy(H):
        return sum(float(np.sum(H.state(l)[lv.leaf_cells()])) * lv.dx ** 3 for l, lv in enumerate(levels))

    out = {"workload": "two-level heat: 64^3 base + 64^3 fine cells on the central 1/8, fine first",
           "coarse_steps": coarse_steps, "use_graph": 3, "check_every": check_every}
    for name, kind, alpha in (("dirichlet", ats.ATS_FACE_DIRICHLET, 1.0), ("neumann", ats.ATS_FACE_NEUMANN, 0.0),
                              ("robin_0.5", ats.ATS_FACE_ROBIN, 0.5)):
        row = {}
        for ug, key in ((3, "ms_per_coarse_step"), (2, "ms_per_coarse_step_deferred")):
            H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
            H.set_interface(kind, alpha)
            for l, (E, K) in enumerate(states):
                H.set_state(l, E, K)
            opts = dict(tol=5e-11, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, use_graph=ug,
                        check_every=check_every)
            H.advance(0, dt, **opts)  # warm-up step (plans, device loops; with 3 the step's capture)
            e0 = energy(H)
            t0 = time.perf_counter()
            for _ in range(coarse_steps):
                code, _ = H.advance(0, dt, **opts)
                if code < 0:  # a warning (ATS_WARN_NEGATIVE) is a result
                    raise RuntimeError(f"amr {name} step failed: {code}")
            t_s = time.perf_counter() - t0
            e1 = energy(H)
            row[key] = round(t_s / coarse_steps * 1e3, 3)
            if ug == 3:
                row["energy_change_per_step"] = float((e1 - e0) / e0 / coarse_steps)
                row["graph"] = H.graph_stats()
            H.close()
        out[name] = row
    return out


def run_fld_amr(ats, ctx, coarse_steps=3):
    """The radiation-matter workload: base 128^3 and three refined levels
    (density above 4^(l+1) x the mean), flux-limited coefficients from each
    level's E^n, linearised gas coupling, fine levels first, mixed precision
    certified to 5e-11 per level solve: time per coarse step (15 level
    solves) as one captured graph (use_graph = 3) and with deferred solves
    (use_graph = 2), and the solve statistics."""
    levels, states, k0, cfl = W.radiation_matter_amr(n0=128)
    rho = [s[1] for s in states]
    kmed = np.median((1.0 / 3.0) / (k0 * rho[0] ** 2))
    dt = cfl * levels[0].dx ** 2 / (2.0 * kmed)
    res = {}
    for ug in (3, 2):
        H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
        try:
            for l, (E, r, t) in enumerate(states):
                H.set_state(l, E, np.ones_like(E))
            for l, (E, r, t) in enumerate(states):
                H.set_fld(l, r, t, k0)
            opts = dict(tol=5e-11, stop_rule=ats.ATS_STOP_CERTIFIED, precision=ats.ATS_PREC_MIXED, use_graph=ug)
            code, st = H.advance(0, dt, **opts)  # warm-up (plans, device loops; with 3 the step's capture)
            if code < 0:
                raise RuntimeError(f"fld warm-up step failed: {code}")
            its = 0
            t0 = time.perf_counter()
            for _ in range(coarse_steps):
                code, st = H.advance(0, dt, **opts)
                if code < 0:  # a warning (ATS_WARN_NEGATIVE) is a result
                    raise RuntimeError(f"fld coarse step failed: {code}")
                its += st["iterations"]
            el = time.perf_counter() - t0
            res[ug] = (el, its, H.graph_stats())
        finally:
            H.close()
    el, its, graph = res[3]
    return {"workload": "4-level AMR radiation-matter: base 128^3 + %s cells, 15 level solves per coarse step, "
                        "fine first" % "/".join(str(lv.n_cell) for lv in levels[1:]),
            "coarse_steps": coarse_steps, "use_graph": 3, "ms_per_coarse_step": round(el / coarse_steps * 1e3, 3),
            "ms_per_coarse_step_deferred": round(res[2][0] / coarse_steps * 1e3, 3), "graph": graph,
            "cg_iterations_per_coarse_step": its / coarse_steps,
            "cells_per_coarse_step": int(sum(lv.n_cell * 2 ** l for l, lv in enumerate(levels)))}


def run_equilibrium(ats, ctx):
    """The equilibrium test with a nonlinear diffusion coefficient (Sect.
    4.2) on uniform grids of 8..128 cells: steps to the steady state (lagged
    K = E^1.5 evaluated on the device, mixed precision, certified 5e-11 per
    step, one graph per solve), the paper's L2 norm against the closed form,
    and its ratio per halving of dx (the paper: close to second order)."""
    from paper_1401_1112_gb300 import equilibrium as G

    rows = []
    for n in (8, 16, 32, 64, 128):
        lv, E, fE, _ = W.equilibrium_column(n)
        Es, steps, ok, s_step = G.relax(ctx, lv, E, fE)
        rows.append({"cells_x": n, "steps": steps, "converged": bool(ok), "ms_per_step": round(s_step * 1e3, 3),
                     "l2": G.l2_error(lv, Es)})
    ratios = [round(rows[i]["l2"] / rows[i + 1]["l2"], 3) for i in range(len(rows) - 1)]
    # the adaptive-time-step runs: base 8 cells, up to four levels refining
    # toward the steep end, fine levels first
    amr = []
    for l_max in range(5):
        levels, E_init, walls = W.equilibrium_amr(l_max)
        Es, steps, ok, s_step = G.relax_amr(ctx, levels, E_init, walls)
        amr.append({"l_max": l_max, "effective_cells_x": 8 * 2 ** l_max, "coarse_steps": steps, "converged": bool(ok),
                    "ms_per_coarse_step": round(s_step * 1e3, 3),
                    "l2": G.l2_error_amr(levels, Es, 8 * 2 ** l_max)})
    return {"workload": "1D column, E = 4 / 0.5 Dirichlet walls, K = E^1.5 lagged, dt = 0.1, to a step change "
                        "< 1e-10", "grids": rows, "l2_ratio_per_halving": ratios, "adaptive": amr}


def run_dirac(ats, ctx, n_steps=64):
    """The linear diffusion (Dirac) test of Sect. 4.1: a pulse of weight 1e5
    on a 1D column (base 32 cells, three levels, effective 256), the mesh
    rebuilt from the 25 % gradient criterion before every coarse step, 64
    coarse steps of 3.125e-15 to t = 2e-13, for each interface row: relative
    change of the total energy and the largest relative error against the
    analytic profile in the pulse's core (|x - x0| < 2 sqrt(2 K t))."""
    from paper_1401_1112_gb300 import amr1d as G

    out = {"workload": "1D pulse, K = 1e10, base 32 cells + 3 levels following the 25% criterion, 64 coarse "
                       "steps to t = 2e-13, mixed precision, certified 5e-11 per solve", "rows": {}}
    t = n_steps * G.COARSE_DT
    for name, kind, alpha in (("dirichlet", ats.ATS_FACE_DIRICHLET, 1.0), ("robin_0.5", ats.ATS_FACE_ROBIN, 0.5),
                              ("neumann", ats.ATS_FACE_NEUMANN, 0.0)):
        levels, E, energies, x0, s_step = G.run_pulse(ctx, kind, alpha, n_steps=n_steps)
        x, dx, e = G.leaf_row(levels, E)
        ref = G.pulse_solution(x, t, x0)
        core = np.abs(x - x0) < 2.0 * np.sqrt(2.0 * G.K_PULSE * t)
        rel = energies / energies[0] - 1.0
        out["rows"][name] = {
            "energy_change_at_steps": {str(k): float(rel[k]) for k in (1, 8, 16, 32, n_steps)},
            "max_rel_error_core": float(np.max(np.abs(e[core] - ref[core]) / ref[core])),
            "finest_level_cells_x": int(np.sum(dx == dx.min())),
            "ms_per_coarse_step": round(s_step * 1e3, 3)}
    return out


def _serve_oracle_check(job):
    """Oracle solution of one served request and its distance to the served
    result: both stop on the residual rule (the served one on ||r|| <= tol
    ||r0||, the oracle to a certified 1e-12), and lambda_min >= 1 bounds each
    solution's distance to the exact one by its residual."""
    (lv, st), x, res_norm = job
    import oracle

    S = oracle.assemble(lv, st.dt, st.K, st.E, face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)
    xr, info = oracle.pcg(S, st.E, tol=1e-12, stop_rule=oracle.STOP_CERTIFIED)
    err = float(np.linalg.norm(x - xr))
    bound = float(res_norm + info["residual"])
    return {"cells": int(lv.n_cell), "abs_err": err, "bound": bound, "rel_err": err / float(np.linalg.norm(xr)),
            "within_bound": bool(err <= 1.0001 * bound + 1e-14 * float(np.linalg.norm(xr)))}


def _build_stream(pool, reqs, ks, window=64):
    """(k, built request) for k in ks, in order, built on the pool's
    processes at most `window` requests ahead of use, so the host holds a
    bounded number of built requests whatever the stream's length."""
    import collections
    import itertools

    it = iter(ks)
    pend = collections.deque((k, pool.apply_async(W.build_request, (reqs[k],))) for k in itertools.islice(it, window))
    while pend:
        k, r = pend.popleft()
        for k2 in itertools.islice(it, 1):
            pend.append((k2, pool.apply_async(W.build_request, (reqs[k2],))))
        yield k, r.get()


def run_serve(args, ats, device):
    """Served request stream (the served workload: Poisson arrivals of level
    solves, cells log-uniform 16^3 .. serve_max_cells, Dirichlet / Neumann /
    Robin walls, tol 1e-6 or 1e-10 on the residual rule; the first
    serve_requests requests of its 2 000).  Requests are built on every host
    core while the stream runs, a bounded number ahead of their arrival (a
    built request is the client's data: the timed service starts at its
    submission).  Then:
      * the plain per-solve FP64 path's service time (level creation,
        operator build and solve, one at a time) on the first up to 240
        requests gives its capacity, and the arrivals are paced at 0.8 x that
        capacity;
      * the continuous-batching server (mixed precision) serves the arrivals,
        with the serve_budget_gb device budget and again with a 4 GB budget
        (admission limited by memory);
      * the plain per-solve FP64 path serves the same arrivals for real: one
        request at a time in arrival order, each started when it has arrived
        and the previous one is done;
      * a sample of served results (the smallest request, a median one and the
        smallest of at least 128^3 cells) is checked against the oracle.
    Reports p50 / p99 latency (submission to result) and throughput."""
    import multiprocessing as mp

    reqs = W.served_requests(n_req=args.serve_requests, seed=1405, hi_cells=args.serve_max_cells)
    n = len(reqs)
    octs = np.array([r["octs"] for r in reqs])
    order = np.argsort(octs)
    sample = {int(order[0]), int(order[n // 2])}
    big = [k for k in order if 8 * octs[k] >= 128 ** 3]
    if big:
        sample.add(int(big[0]))
    kept = {}

    def fp64_serve_one(ctx, built, tol):
        lv, st = built
        L = ats.Level(ctx, lv)
        L.build(st.dt, st.K, st.E, face_E=st.face_E, face_F=st.face_F)
        x = st.E.copy()
        code, _ = L.solve(x, tol=tol, precision=ats.ATS_PREC_FP64)
        L.close()
        if code < 0:  # a warning (ATS_WARN_NEGATIVE) is a result
            raise RuntimeError("fp64 served solve failed")

    cores = max(1, (os.cpu_count() or 2) - 2)
    with mp.get_context("spawn").Pool(cores) as pool:
        # plain per-solve FP64: service time of the first requests (level, build, solve)
        n_cal = min(n, 240)
        svc = []
        with ats.Context(device) as ctx:
            for k, b in _build_stream(pool, reqs, range(n_cal)):
                if k == 0:
                    fp64_serve_one(ctx, b, reqs[k]["tol"])  # warm-up
                t0 = time.perf_counter()
                fp64_serve_one(ctx, b, reqs[k]["tol"])
                svc.append(time.perf_counter() - t0)
        svc = np.array(svc)
        cap = len(svc) / svc.sum()
        lam = 0.8 * cap
        arrivals = np.array([r["t"] for r in reqs]) * (reqs[-1]["id"] + 1) / reqs[-1]["t"] / lam

        def server_run(budget_bytes, keep):
            srv = ats.Server(device, mem_budget_bytes=int(budget_bytes), precision=ats.ATS_PREC_MIXED,
                             check_every=4)
            tickets = [None] * n
            n_cell = [0] * n
            cells = [0]
            t_start = time.perf_counter()

            def submitter():
                for k, (lv, st) in _build_stream(pool, reqs, range(n)):
                    delay = arrivals[k] - (time.perf_counter() - t_start)
                    if delay > 0:
                        time.sleep(delay)
                    n_cell[k] = lv.n_cell
                    cells[0] += lv.n_cell
                    if k in keep:
                        kept[k] = (lv, st)
                    tickets[k] = srv.submit(lv, st, tol=reqs[k]["tol"])

            th = threading.Thread(target=submitter)
            th.start()
            lat, xs, rn = [], {}, {}
            errs = 0
            for k in range(n):
                while tickets[k] is None:
                    time.sleep(0.0002)
                code, x, res = srv.wait(tickets[k], n_cell[k])
                errs += code < 0
                lat.append(res["latency_us"] / 1e3)
                if k in keep:
                    xs[k] = x
                    rn[k] = res["stats"]["res_norm"]
            t_end = time.perf_counter()
            th.join()
            st_srv = srv.stats()
            srv.close()
            lat = np.array(lat)
            return {"throughput": round(n / (t_end - t_start), 2), "unit": UNIT,
                    "p50_ms": round(float(np.percentile(lat, 50)), 3),
                    "p99_ms": round(float(np.percentile(lat, 99)), 3),
                    "errors": int(errs), "peak_resident": st_srv["peak_resident"],
                    "budget_gb": round(budget_bytes / (1 << 30), 1), "cells_mean": round(cells[0] / n)}, xs, rn

        served, xs, rn = server_run(args.serve_budget_gb * (1 << 30), sample)
        served_small, _, _ = server_run(4 * (1 << 30), set())

        # the plain per-solve FP64 path serving the same arrivals, one at a time
        fin = np.zeros(n)
        with ats.Context(device) as ctx:
            t_start = None
            for k, b in _build_stream(pool, reqs, range(n)):
                if t_start is None:
                    fp64_serve_one(ctx, b, reqs[k]["tol"])  # warm-up
                    t_start = time.perf_counter()
                delay = arrivals[k] - (time.perf_counter() - t_start)
                if delay > 0:
                    time.sleep(delay)
                fp64_serve_one(ctx, b, reqs[k]["tol"])
                fin[k] = time.perf_counter() - t_start
            t_end = time.perf_counter()
        lat64 = (fin - arrivals) * 1e3

    checks = []
    if not args.no_cpu:
        with mp.get_context("spawn").Pool(max(1, len(sample))) as pool:
            checks = pool.map(_serve_oracle_check, [(kept[k], xs[k], rn[k]) for k in sorted(sample)], chunksize=1)

    return {
        "requests": n, "of": 2000, "max_cells": int(args.serve_max_cells),
        "arrival_rate_per_s": round(lam, 2), **served,
        "budget_4gb": served_small,
        "fp64_per_solve": {"capacity": round(cap, 2), "capacity_sample": int(n_cal),
                           "throughput": round(n / (t_end - t_start), 2),
                           "p50_ms": round(float(np.percentile(lat64, 50)), 3),
                           "p99_ms": round(float(np.percentile(lat64, 99)), 3),
                           "path": "plain per-solve FP64 (level, build, solve), one request at a time in arrival "
                                   "order on the same arrivals"},
        "oracle_check": checks,
    }


# ---------------------------------------------------------------------------
# oracle (CPU) arm
# ---------------------------------------------------------------------------

def _oracle_warm(_):
    import oracle  # noqa: F401  (loads the compiled oracle in the worker)

    return os.getpid()


def _oracle_solve(job):
    lv, st = job
    import oracle

    S = oracle.assemble(lv, st.dt, st.K, st.E, face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)
    oracle.pcg(S, st.E, tol=TOL, stop_rule=oracle.STOP_CERTIFIED)
    return lv.n_cell


def oracle_all_cores(jobs, cores=None):
    """The same oracle solves spread over every host core (one spawned
    process per core, started and warmed before the clock starts; each solve
    is sent to a worker and solved there): solves per second of wall time."""
    import multiprocessing as mp

    cores = cores or os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_warm, range(cores), chunksize=1)
        # largest first, one at a time: the workers stay evenly loaded
        jobs = sorted(jobs, key=lambda j: -j[0].n_cell)
        t0 = time.perf_counter()
        cells = sum(pool.imap_unordered(_oracle_solve, jobs, chunksize=1))
        el = time.perf_counter() - t0
    return {"value": round(len(jobs) / el, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the same {len(jobs)} solves ({cells} cells) on {cores} worker processes, {el:.1f} s"}


def cpu_baseline(solves, budget_s=15.0, seed=7, gpu_results=None, all_cores=True):
    """The FP64 CPU oracle as it stands (assembly + Jacobi-PCG to the same
    tolerance) on a random sample of the same solves, until ~budget_s.
    gpu_results: {path: [x per solve]} of GPU solutions of the same solves;
    the relative L2 difference of each to the oracle's solution of every
    sampled solve is reported (max and median per path)."""
    import oracle

    rng = np.random.default_rng(seed)
    order = rng.permutation(len(solves))
    t0 = time.perf_counter()
    done = 0
    cells = 0
    errs = {k: [] for k in (gpu_results or {})}
    timed = 0.0
    for k in order:
        lv, st = solves[k]
        t1 = time.perf_counter()
        S = oracle.assemble(lv, st.dt, st.K, st.E, face_K=st.face_K, face_E=st.face_E, face_F=st.face_F)
        xr, _ = oracle.pcg(S, st.E, tol=TOL, stop_rule=oracle.STOP_CERTIFIED)
        timed += time.perf_counter() - t1
        for path, xs in (gpu_results or {}).items():
            errs[path].append(float(np.linalg.norm(xs[k] - xr) / np.linalg.norm(xr)))
        done += 1
        cells += lv.n_cell
        if time.perf_counter() - t0 >= budget_s:
            break
    out = {"value": round(done / timed, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{done} of {len(solves)} solves drawn at random ({cells} cells), FP64 assembly + Jacobi-PCG "
                     f"to ||b - Ax|| <= 5e-11 ||x||, single thread, {timed:.1f} s"}
    if all_cores:
        out["all_cores"] = oracle_all_cores([solves[k] for k in order[:done]])
    if errs:
        out["error_vs_oracle"] = {
            path: {"max_rel_l2": float(np.max(v)), "median_rel_l2": float(np.median(v)), "solves": len(v)}
            for path, v in errs.items()}
    return out


def run_configs(ats, ctx):
    """Every workload configuration timed the same way on the oracle (one
    host thread, the cpu_baseline of that configuration) and on the GPU (FP64
    and mixed, after a warm-up), each solve certified to 5e-11, with the GPU
    result's relative L2 difference to the oracle's:
      gaussian_32cube: one level, 32^3 Gaussian, one step;
      two_level_64cube: two levels, 64^3 + 64^3 central, one coarse step (coarse first, fine
         ghosts linear in time);
      radiation_matter_128cube: four levels, radiation-matter, base 128^3, one coarse step (fine
         first).
    (The batched and served configurations are the main line and its serve
    leg.)"""
    import oracle
    from oracle import driver

    out = {}
    opts = dict(tol=5e-11, stop_rule=ats.ATS_STOP_CERTIFIED, use_graph=2)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    # one level, 32^3 Gaussian
    lv, st = W.gaussian_32cube(32)
    t0 = time.perf_counter()
    S = oracle.assemble(lv, st.dt, st.K, st.E)
    xr, info = oracle.pcg(S, st.E, tol=5e-11, stop_rule=oracle.STOP_CERTIFIED)
    t_or = time.perf_counter() - t0
    L = ats.Level(ctx, lv)
    row = {"cells": lv.n_cell, "oracle_ms": round(t_or * 1e3, 3), "iterations": info["iterations"]}
    for name, prec in (("fp64", ats.ATS_PREC_FP64), ("mixed", ats.ATS_PREC_MIXED)):
        L.build(st.dt, st.K, st.E)
        x = st.E.copy()
        L.solve(x, precision=prec, **opts)
        t0 = time.perf_counter()
        reps = 20
        for _ in range(reps):
            L.build(st.dt, st.K, st.E)
            x = st.E.copy()
            code, _ = L.solve(x, precision=prec, **opts)
        row[name + "_ms"] = round((time.perf_counter() - t0) / reps * 1e3, 3)
        row[name + "_rel_l2_vs_oracle"] = rel(x, xr)
    L.close()
    out["gaussian_32cube"] = row

    # two levels, 64^3 + 64^3, coarse first (the reading of the linear-in-time ghost)
    levels, states, dt = W.two_level_gaussian_64cube(64)
    ref = driver.Hierarchy(levels, states, order="coarse_first")
    t0 = time.perf_counter()
    ref.advance(0, dt, tol=5e-11)
    t_or = time.perf_counter() - t0
    row = {"cells": int(sum(lv.n_cell for lv in levels)), "oracle_ms": round(t_or * 1e3, 1)}
    for name, prec in (("fp64", ats.ATS_PREC_FP64), ("mixed", ats.ATS_PREC_MIXED)):
        H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_COARSE_FIRST)
        for l, (E, K) in enumerate(states):
            H.set_state(l, E, K)
        H.advance(0, dt, precision=prec, **opts)  # plans and graphs; the timed step is the same step again
        for l, (E, K) in enumerate(states):
            H.set_state(l, E, K)
        t0 = time.perf_counter()
        H.advance(0, dt, precision=prec, **opts)
        row[name + "_ms"] = round((time.perf_counter() - t0) * 1e3, 3)
        row[name + "_rel_l2_vs_oracle"] = max(rel(H.state(l), ref.state(l)) for l in range(len(levels)))
        H.close()
    out["two_level_64cube"] = row

    # four levels, radiation-matter, base 128^3
    levels, states, k0, cfl = W.radiation_matter_amr(n0=128)
    rho = [s_[1] for s_ in states]
    T = [s_[2] for s_ in states]
    kmed = np.median((1.0 / 3.0) / (k0 * rho[0] ** 2))
    dt = cfl * levels[0].dx ** 2 / (2.0 * kmed)
    ref = driver.Hierarchy(levels, [(E, np.ones_like(E)) for E, _, _ in states], order="fine_first",
                           fld=([r.copy() for r in rho], [t_.copy() for t_ in T], k0))
    t0 = time.perf_counter()
    ref.advance(0, dt, tol=5e-11)
    t_or = time.perf_counter() - t0
    row = {"cells": int(sum(lv.n_cell for lv in levels)), "oracle_ms": round(t_or * 1e3, 1)}
    for name, prec in (("fp64", ats.ATS_PREC_FP64), ("mixed", ats.ATS_PREC_MIXED)):
        H = ats.Hierarchy(ctx, levels, ats.ATS_ORDER_FINE_FIRST)
        for timed in (False, True):  # a warm-up step (plans, graphs), then the same step again
            for l, (E, r, t) in enumerate(states):
                H.set_state(l, E, np.ones_like(E))
            for l, (E, r, t) in enumerate(states):
                H.set_fld(l, r, t, k0)
            t0 = time.perf_counter()
            H.advance(0, dt, precision=prec, **opts)
            el = time.perf_counter() - t0
        row[name + "_ms"] = round(el * 1e3, 3)
        row[name + "_rel_l2_vs_oracle"] = max(rel(H.state(l), ref.state(l)) for l in range(len(levels)))
        H.close()
    out["radiation_matter_128cube"] = row
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    solves = W.ragged_batch(n_solves=args.solves, seed=1404)
    import multiprocessing as mp

    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    per_step = args.ref_solves_per_step or 12 * cores
    rng = np.random.default_rng(11)
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_warm, range(cores), chunksize=1)

        def step():
            idx = rng.choice(len(solves), size=min(per_step, len(solves)), replace=False)
            jobs = sorted((solves[k] for k in idx), key=lambda j: -j[0].n_cell)  # largest first
            for _ in pool.imap_unordered(_oracle_solve, jobs, chunksize=1):
                pass

        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        el = time.perf_counter() - t0
    v = per_step * args.steps / el
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * el / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"batched level solves: {args.solves} ragged single-level backward-Euler solves, "
                               f"8^3..64^3 cells, FP64 CPU oracle to ||b - Ax|| <= 5e-11 ||x||, {per_step} random "
                               f"solves per step on {cores} worker processes",
                   "solves": args.solves, "tol": TOL, "seed": 1404},
        "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} random solves of the {args.solves}-solve batch per step, one "
                                   f"process per core"},
        "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--solves", type=int, default=512)
    ap.add_argument("--check-every", type=int, default=16)
    ap.add_argument("--tile", type=int, default=0, help="octs per work item (0 = library default)")
    ap.add_argument("--inner-rtol", type=float, default=0.0, help="mixed inner reduction (0 = library default)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-solves-per-step", type=int, default=0, help="0 = twelve per host core")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-amr", action="store_true")
    ap.add_argument("--no-cn", action="store_true")
    ap.add_argument("--no-equilibrium", action="store_true")
    ap.add_argument("--no-dirac", action="store_true")
    ap.add_argument("--no-fld", action="store_true")
    ap.add_argument("--configs", action="store_true",
                    help="time each workload configuration on the oracle and the GPU (one JSON line) instead")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--res-max-octs", type=int, default=32768,
                    help="levels up to this many octs take the resident solver (0 = the library default)")
    ap.add_argument("--cg-form", type=int, default=0,
                    help="resident CG step: 1 = q from p after a group barrier, 2 = q by recurrence (0 = default)")
    ap.add_argument("--serve-requests", type=int, default=240,
                    help="requests of the served stream's 2 000 (the first N, same arrival process)")
    ap.add_argument("--serve-max-cells", type=int, default=256 ** 3)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    args = ap.parse_args()
    rank, world, local = _dist()
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist

        dist.init_process_group(backend="nccl")
    if args.configs:
        if rank != 0:
            return
        import torch

        from paper_1401_1112_gb300 import ats, build

        build.build()
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        with ats.Context(0) as ctx:
            ctx.set_stream(stream.cuda_stream)
            print(json.dumps({"configs": run_configs(ats, ctx)}), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
