"""Benchmark: (design . k) band + adjoint solves per second on the FCC primitive cell with
729 plane waves, 20 bands and 100 k-points per design (32^3 voxels, seeded level-set
designs, WC / epoxy, SIMP p = 3).

One step = one design evaluation through the C ABI: pc_set_design (SIMP fields,
structure factors, Toeplitz operators, inverse compliance blocks), pc_bands (batched
block eigensolver over all 100 k + FP64 Rayleigh-Ritz) and pc_gap_and_grad in the
all-band weighted form (every (k, band) carries a weight, so the adjoint work is the
full per-(design . k) work).  The mixed-precision form is the headline; the plain FP64
GPU form is timed beside it.  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "design·k band+adjoint solves/s (FCC, N=729, 20 bands) mixed vs FP64; % roofline"
UNIT = "(design*k)/s"
BENCH_WORKLOAD = "fcc32_M4_levelset"
WORKLOAD = "fcc32_M4_levelset: FCC primitive cell, 32^3 voxels, N=729 plane waves, 100 k, 20 bands"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--cpu-k", type=int, default=2, help="k-points in the oracle sample")
    ap.add_argument("--workload", default=BENCH_WORKLOAD,
                    choices=["sc16_M2_grf", "bcc24_M3_grf", BENCH_WORKLOAD, "batch32_mixed", "sphere_scan"],
                    help="the FCC N = 729 workload is the benchmark; sc16/bcc24 are smaller cases for "
                         "profiler captures; batch32_mixed (32 designs of uneven lattice and N in one "
                         "call) and sphere_scan (the paper's sphere-inclusion volume-fraction scans) "
                         "are the batch workloads")
    return ap.parse_args()


def designs(count: int, rank: int, workload: str = BENCH_WORKLOAD):
    gen = wl.WORKLOADS[workload]
    return [gen(design=rank * 1000 + i) for i in range(count)]


def replica_max(ms_step: float, world: int, device) -> float:
    """Slowest rank's step time: every rank runs its own designs (independent replicas, no
    data exchange), so the job's step ends when the last rank's does."""
    if world == 1:
        return ms_step
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_step], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ms_step: float, nk: int, world: int) -> float:
    """Whole-job (design*k)/s: world ranks each finish one nk-point design per ms_step."""
    return world * nk / (ms_step * 1e-3)


def all_band_weights(w):
    """Dense positive weights on every (k, band) except the Gamma zero modes."""
    wt = np.full((w.nk, w.nbands), 1.0 / (w.nk * w.nbands))
    for k in range(w.nk):
        if np.allclose(w.Q[k], 0.0):
            wt[k, :3] = 0.0
    return wt


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(nk_sample: int):
    """The FP64 oracle (as it stands) on one FCC N = 729 design: per-design assembly and
    Phi^-1 once, then nk_sample wavevectors with their all-band adjoint.  The per
    (design . k) time is extrapolated to the 100-k design: (t_design + 100 t_k) / 100."""
    from oracle import mixed, sensitivity
    w = wl.fcc32_levelset(design=0)
    t0 = time.perf_counter()
    P = mixed.from_workload(w)
    P.phi_inv()
    t1 = time.perf_counter()
    wts = all_band_weights(w)
    ks = np.linspace(1, w.nk - 1, nk_sample).astype(int)
    grad = np.zeros(w.rho.size)
    for k in ks:
        sol = mixed.solve_k(P, w.Q[k], w.nbands, literal=False)
        for b in range(w.nbands):
            grad += wts[k, b] * sensitivity.voxel(P, sol.lam[b], sol.theta[:, b], sol.s[:, b])
    t2 = time.perf_counter()
    assert np.isfinite(grad).all()
    t_design, t_k = t1 - t0, (t2 - t1) / len(ks)
    per = (t_design + w.nk * t_k) / w.nk
    cores = len(os.sched_getaffinity(0))
    return {"value": 1.0 / per, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"1 design (assembly + Phi^-1: {t_design:.1f} s) and {len(ks)} of 100 k-points "
                      f"({t_k:.1f} s each incl. 20-band adjoint); extrapolated to the 100-k design",
            "seconds": t2 - t0}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    total = args.warmup + args.steps
    vals = []
    for i in range(total):
        r = cpu_baseline(1)
        if i >= args.warmup:
            vals.append(r)
    value = float(np.mean([v["value"] for v in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * 100 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"kind": "oracle", "cores": vals[0]["cores"], "sample": vals[0]["sample"], "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# DRAM traffic per launch of the dominant kernels, from one ncu capture each (dram__bytes_read.sum +
# dram__bytes_write.sum; the summaries are under profiles/).  Each entry holds the SHA-256 of the
# kernel's source file when it was captured: once that file changes, the figure is stale and the
# bench reports null.
TRAFFIC = {  # DRAM bytes (read + write) per launch from ncu, single-stream pass of the FCC N = 729 workload
    "k_tc_gram": {"source": "tall_tc.cu", "sha256": "78378b59f258febe9197fcc58c746a92767b5607aaf550d16906971e3962b04e", "bytes": 1.841e+08},
    "k_tc_update": {"source": "tall_tc.cu", "sha256": "78378b59f258febe9197fcc58c746a92767b5607aaf550d16906971e3962b04e", "bytes": 2.772e+08},
    "k_tc_gemm": {"source": "gemm_tc.cu", "sha256": "2c173663d760f16a1c803e148a9ef5a7323bdd3c7c262b5b58d0381bed90268f", "bytes": 3.159e+08},
    "k_small_rr32": {"source": "small_rr.cu", "sha256": "caf29f36352a8d6c949bef63ca800f9978062abb8d790cd4568ff6464c5b4abb", "bytes": 7.744e+06},
    "k_oz_gemm": {"source": "oz_gemm.cu", "sha256": "79dba0c8329328bf1c050d62d0a79c5b981615f008545982d8e2c97b98c3e863", "bytes": 2.75e+08},
    "k_adj_synth12+k_adj_reduce": {"source": "adjoint.cu", "sha256": "997172643ab95aec17220765c988d0909ce1bba69a3b1003d49f11ec7982849f", "bytes": 1.398e+09},
}


def traffic_per_launch(kernel: str):
    t = TRAFFIC.get(kernel)
    if not t:
        return None
    import hashlib
    path = os.path.join(ROOT, "paper_1603_06855_gb300", "csrc", t["source"])
    try:
        sha = hashlib.sha256(open(path, "rb").read()).hexdigest()
    except OSError:
        return None
    return t["bytes"] if sha == t["sha256"] else None


def measured_peaks() -> dict:
    """HBM copy bandwidth and bf16 GEMM throughput measured on this GPU pool (JSON at the repo root)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def run_batch(args, dev, rank, world, barrier):
    """Batch workloads through the one-call interface (pc_batch_*): one step = set_designs, bands
    and gap_and_grad of every design (all-band weights for batch32_mixed, gap(6,7) for the scans)."""
    import torch
    from paper_1603_06855_gb300 import autotune
    from paper_1603_06855_gb300 import binding as B
    from paper_1603_06855_gb300.solver import BatchSolver
    designs = wl.batch32_mixed() if args.workload == "batch32_mixed" else wl.sphere_scan()
    dk = sum(len(w.Q) for w in designs)
    rhos = [w.rho for w in designs]
    props = torch.cuda.get_device_properties(dev)
    t_tune = time.perf_counter()
    workers, kgroups = autotune.choose(designs, B.PC_MIXED, rhos, autotune.measure_batch, props.name,
                                       props.multi_processor_count)
    t_tune = time.perf_counter() - t_tune
    allband = args.workload == "batch32_mixed"

    def evaluate(bs, ds, rh, wt):
        bs.set_designs(rh)
        oms = bs.bands()
        if allband:
            gaps, _ = bs.gap_and_grad(mode=B.PC_GRAD_ALLBANDS, weights=wt)
        else:
            gaps, _ = bs.gap_and_grad(n_lower=[6] * len(ds))
        return oms, gaps

    def timed(bs, ds, steps, warmup):
        rh = [w.rho for w in ds]
        wt = [torch.from_numpy(all_band_weights(w)) for w in ds] if allband else None
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        for i in range(warmup):
            evaluate(bs, ds, rh, wt)
        torch.cuda.synchronize(dev)
        launches0 = bs.stats(0).launches  # the library's launch counter is process-wide
        clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
        barrier()
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        out = None
        for i in range(steps):
            flush.fill_(float(i))
            torch.cuda.synchronize(dev)
            e0.record()
            out = evaluate(bs, ds, rh, wt)
            e1.record()
            torch.cuda.synchronize(dev)
            ms += e0.elapsed_time(e1)
        barrier()
        ck = clocks.stop()
        return ms / steps, ck, out, bs.stats(0).launches - launches0

    bs = BatchSolver(designs, B.PC_MIXED, workers=workers, kgroups=kgroups)
    ms, ck, (oms, gaps), launches = timed(bs, designs, args.steps, args.warmup)
    for d in range(len(designs)):
        st = bs.stats(d)
        if st.status != B.PC_OK:
            raise RuntimeError(f"{designs[d].name}: {B.pc_strerror(st.status)}")
    bs.close()
    ms_step = replica_max(ms, world, dev)
    value = world * dk / (ms_step * 1e-3)
    # the same batch one design at a time (one worker, the contexts' own k groups)
    seq = BatchSolver(designs, B.PC_MIXED, workers=1, kgroups=0)
    ms_seq, _, _, _ = timed(seq, designs, 1, 1)
    seq.close()
    line = {"metric": f"design·k band+adjoint solves/s ({args.workload}, one batch call)", "value": value,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 block iteration (split-bf16x3 tensor-core contractions, f32 projected problems) + f64 Rayleigh-Ritz",
            "data": "synthetic",
            "config": {"workload": args.workload, "designs": len(designs), "design_k_per_step": dk,
                       "adjoint": "all-band weighted" if allband else "gap(6,7)",
                       "batch_workers": workers, "batch_kgroups": kgroups, "autotune_seconds": t_tune,
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "clocks": ck, "gpu_launches": int(launches),
            "one_design_at_a_time": {"value": dk / (ms_seq * 1e-3), "unit": UNIT, "ms": ms_seq}}
    if allband and not args.no_fp64:
        # the plain FP64 GPU form per design on one design per (lattice, N) bucket, 8 k-points
        # each, beside the mixed form per design on the same subset
        pick = {}
        for i, w in enumerate(designs):
            pick.setdefault((w.lattice, (2 * w.M + 1) ** 3), i)
        sub = []
        for i in pick.values():
            w = designs[i]
            sub.append(wl.Workload(w.name, w.lattice, w.n, w.M, w.nbands, w.Q[:8], w.rho, w.penal, w.gaps, w.seed))
        res = {}
        for prec, name in ((B.PC_FP64, "fp64"), (B.PC_MIXED, "mixed")):
            sb = BatchSolver(sub, prec, workers=1, kgroups=0)
            ms_s, _, _, _ = timed(sb, sub, 1, 1)
            sb.close()
            res[name] = sum(len(w.Q) for w in sub) / (ms_s * 1e-3)
        line["fp64_form"] = {"value": res["fp64"], "unit": UNIT, "subset": f"{len(sub)} designs (one per "
                             "lattice x N bucket), 8 k-points each, one design at a time",
                             "mixed_same_subset": res["mixed"], "mixed_over_fp64": res["mixed"] / res["fp64"]}
    if not allband:
        best = {}
        for w, g in zip(designs, gaps.cpu().numpy()):
            lat, vf = w.lattice, float(w.name.split("vf")[1])
            if lat not in best or g > best[lat][0]:
                best[lat] = (float(g), vf)
        line["scan_maxima"] = {lat: {"gap_pct": 100 * g, "volume_fraction": vf} for lat, (g, vf) in best.items()}
        line["scan_maxima_printed"] = {"sc": [67.5, 0.412], "bcc": [94.2, 0.545], "fcc": [93.3, 0.588]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    from paper_1603_06855_gb300 import binding as B
    from paper_1603_06855_gb300 import build_lib
    from paper_1603_06855_gb300.solver import BandSolver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build_lib.build()
    B.load()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    if args.workload in ("batch32_mixed", "sphere_scan"):
        run_batch(args, dev, rank, world, barrier)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    nsteps = args.warmup + args.steps
    ws = designs(min(nsteps, 4), rank, args.workload)
    w0 = ws[0]
    rhos = [torch.from_numpy(w.rho.ravel()).to(dev) for w in ws]
    wts = torch.from_numpy(all_band_weights(w0)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def run(precision, steps, warmup, profile=False):
        s = BandSolver.from_workload(w0, precision=precision, device=dev)
        omega = torch.empty((w0.nk, w0.nbands), dtype=torch.float64, device=dev)
        gap = torch.empty(1, dtype=torch.float64, device=dev)
        grad = torch.empty(w0.n, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev)

        def step(i):
            flush.fill_(float(i))
            s.set_design(rhos[i % len(rhos)])
            s.bands(out=omega)
            s.gap_and_grad(mode=B.PC_GRAD_ALLBANDS, weights=wts, gap_out=gap, grad_out=grad)

        for i in range(warmup):
            step(i)
        torch.cuda.synchronize(dev)
        st0 = s.stats()
        if st0.status not in (B.PC_OK,):
            raise RuntimeError(f"warm-up status {B.pc_strerror(st0.status)}")
        B.pc_clear_status(s.ctx)
        if profile:
            B.pc_set_profiling(s.ctx, True)
        clocks = ClockSampler(local)
        barrier()
        torch.cuda.synchronize(dev)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            step(warmup + i)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ck = clocks.stop()
        ms = e0.elapsed_time(e1)
        st = s.stats()
        run.last = ((warmup + steps - 1) % len(rhos), omega, grad)
        return s, ms, st, ck

    # ---- mixed form (headline) ----
    s_mx, ms_mx, st_mx, ck = run(B.PC_MIXED, args.steps, args.warmup, profile=False)
    ms_step = replica_max(ms_mx / args.steps, world, dev)
    value = replica_throughput(ms_step, w0.nk, world)

    # ---- end to end: host buffers, copies inside the timed region ----
    rho_h = [torch.from_numpy(w.rho.ravel()).pin_memory() for w in ws]
    om_h = torch.empty((w0.nk, w0.nbands), dtype=torch.float64).pin_memory()
    gap_h = torch.empty(1, dtype=torch.float64).pin_memory()
    grad_h = torch.empty(w0.n, dtype=torch.float64).pin_memory()
    rho_d = torch.empty(w0.rho.size, dtype=torch.float64, device=dev)
    om_d = torch.empty((w0.nk, w0.nbands), dtype=torch.float64, device=dev)
    gap_d = torch.empty(1, dtype=torch.float64, device=dev)
    grad_d = torch.empty(w0.n, dtype=torch.float64, device=dev)

    def e2e_step(i):
        rho_d.copy_(rho_h[i % len(rho_h)], non_blocking=True)
        B.pc_set_design(s_mx.ctx, rho_d.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
        s_mx.bands(out=om_d)
        s_mx.gap_and_grad(mode=B.PC_GRAD_ALLBANDS, weights=wts, gap_out=gap_d, grad_out=grad_d)
        om_h.copy_(om_d, non_blocking=True)
        gap_h.copy_(gap_d, non_blocking=True)
        grad_h.copy_(grad_d, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()

    e2e_step(0)
    barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        e2e_step(i)
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / args.steps
    e2e_value = world * w0.nk / (e2e_ms * 1e-3)
    h2d = w0.rho.size * 8
    d2h = (w0.nk * w0.nbands + 1 + w0.rho.size) * 8

    # ---- per-phase device times and rooflines: a separate, untimed profiling pass ----
    # The timed run overlaps two halves of the k-points on two streams, so event times of one
    # kernel family include time shared with the other half's kernels.  The kernel families are
    # therefore timed in a single-stream pass (PC_SPLIT=0) of the same workload.
    prof_steps = 2
    os.environ["PC_SPLIT"] = "0"
    try:
        s_pf, ms_pf, st_pf, _ = run(B.PC_MIXED, prof_steps, 1, profile=True)
        s_pf.close()
    finally:
        del os.environ["PC_SPLIT"]

    # ---- roofline of each modelled kernel family; the one with the largest share is reported ----
    fp64_peak = B.pc_probe(0)
    fp32_peak = B.pc_probe(1)
    peaks = measured_peaks()
    steps_ = args.steps
    fam = {}

    def add(name, kernel, ms, amount, launches, bound, peak, unit, source):
        if ms <= 0 or peak is None or amount <= 0:
            return
        achieved = amount / (ms * 1e-3) / (1e12 if unit == "TFLOP/s" else 1e9)
        fam[name] = {"bound": bound, "kernel": kernel, "achieved": achieved, "peak": peak, "unit": unit,
                     "frac": achieved / peak, "traffic": traffic_per_launch(kernel), "peak_source": source,
                     "launches_timed": int(launches), "share_of_step": ms / ms_pf}
        if unit == "GB/s" and launches > 0:  # the algorithmic bytes that traffic is compared with
            fam[name]["algorithmic_bytes_per_launch"] = amount / launches

    # Gram products and basis updates: split-BF16 tensor-core kernels that read each FP32 operand
    # once and write the result once, so HBM bound (algorithmic bytes / measured copy bandwidth)
    if peaks.get("hbm_gbs"):
        add("gram_AhB", "k_tc_gram", st_pf.ms_gram, st_pf.gram_bytes, st_pf.gram_launches, "hbm", peaks["hbm_gbs"],
            "GB/s", "MEASURED_PEAKS.json hbm_gbs")
        add("basis_update_SC", "k_tc_update", st_pf.ms_update, st_pf.update_bytes, st_pf.update_launches, "hbm",
            peaks["hbm_gbs"], "GB/s", "MEASURED_PEAKS.json hbm_gbs")
    # operator apply: split-BF16 tensor-core GEMM; the method's flops against the raw sustained
    # BF16 peak, and beside it against that peak / 6 (six bf16 slice products per FP32-accurate one)
    if peaks.get("bf16_tflops_sustained"):
        add("iteration_operator_apply", "k_tc_gemm", st_pf.ms_iter_apply, st_pf.iter_apply_flops,
            st_pf.iter_apply_calls, "tensor", peaks["bf16_tflops_sustained"], "TFLOP/s",
            "MEASURED_PEAKS.json bf16_tflops_sustained")
        if "iteration_operator_apply" in fam:
            f = fam["iteration_operator_apply"]
            f["frac_of_split_bf16_peak"] = f["achieved"] / (peaks["bf16_tflops_sustained"] / 6.0)
    # final Rayleigh-Ritz operator products: exact 6-bit slice products on the tensor cores (36 bf16
    # products per FP64-accurate one) where the plan fits, else the FP64 CUDA-core GEMM
    if st_pf.rr_sliced and peaks.get("bf16_tflops_sustained"):
        add("fp64_rayleigh_ritz_gemm", "k_oz_gemm", st_pf.ms_rr_gemm, 36.0 * st_pf.rr_gemm_flops,
            st_pf.rr_gemm_launches, "tensor", peaks["bf16_tflops_sustained"], "TFLOP/s",
            "MEASURED_PEAKS.json bf16_tflops_sustained")
        if "fp64_rayleigh_ritz_gemm" in fam:
            f = fam["fp64_rayleigh_ritz_gemm"]
            f["fp64_equivalent_tflops"] = f["achieved"] / 36.0
            f["fp64_equivalent_over_fp64_fma_peak"] = f["achieved"] / 36.0 / (fp64_peak / 1e3)
    else:
        add("fp64_rayleigh_ritz_gemm", "k_gemm<double>", st_pf.ms_rr_gemm, st_pf.rr_gemm_flops,
            st_pf.rr_gemm_launches, "alu", fp64_peak / 1e3, "TFLOP/s",
            "measured FP64 FMA throughput (pc_probe) on this GPU")
    # projected eigenproblems (Cholesky, reduction, Jacobi sweeps as executed) against FP32 FMA; the
    # family time also holds the small Cholesky-QR and conjugate-direction kernels
    add("projected_problems", "k_small_rr32", st_pf.ms_small, st_pf.small_flops, st_pf.small_calls, "alu", fp32_peak / 1e3,
        "TFLOP/s", "measured FP32 FMA throughput (pc_probe) on this GPU")
    # adjoint synthesis and reduction (FP32 in the mixed form)
    add("adjoint", "k_adj_synth12+k_adj_reduce", st_pf.ms_grad_kernels,
        prof_steps * st_pf.grad_pairs * st_pf.grad_flops_per_pair, 2 * prof_steps, "alu", fp32_peak / 1e3,
        "TFLOP/s", "measured FP32 FMA throughput (pc_probe) on this GPU")
    dom = max(fam, key=lambda k: fam[k]["share_of_step"])
    roofline = dict(fam[dom])
    roofline["of"] = "measured"
    roofline["timed_in"] = f"single-stream profiling pass, {prof_steps} steps ({ms_pf / prof_steps:.1f} ms per step)"
    # ---- plain FP64 GPU form ----
    fp64 = None
    if not args.no_fp64 and args.fp64_steps > 0:
        s64, ms64, st64, _ = run(B.PC_FP64, args.fp64_steps, 1, profile=True)
        v64 = w0.nk / (ms64 / args.fp64_steps * 1e-3)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / args.fp64_steps, "iterations": st64.iterations,
                "mixed_over_fp64": value / world / v64}
        # accuracy of the headline form: mixed and FP64 frequencies of the same design (untimed);
        # relative to max(w_fp64, 0.05 max w_fp64), Gamma zero modes (w < 1e-4 max w) left out
        d64, om64, g64 = run.last
        om_mx = torch.empty_like(om64)
        g_mx = torch.empty_like(g64)
        gap_mx = torch.empty(1, dtype=torch.float64, device=dev)
        s_mx.set_design(rhos[d64])
        s_mx.bands(out=om_mx)
        s_mx.gap_and_grad(mode=B.PC_GRAD_ALLBANDS, weights=wts, gap_out=gap_mx, grad_out=g_mx)
        torch.cuda.synchronize(dev)
        fp64["grad_rel_l2_mixed_vs_fp64"] = float(torch.linalg.norm(g_mx - g64) / torch.linalg.norm(g64))
        a, b = om_mx.cpu().numpy(), om64.cpu().numpy()
        err = np.abs(a - b) / np.maximum(b, 0.05 * b.max())
        err[b < 1e-4 * b.max()] = 0.0
        fp64["omega_max_rel_err_mixed_vs_fp64"] = float(err.max())
        fp64["omega_compared"] = f"design {d64}, {b.size} (k, band) pairs"
        s64.close()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 block iteration (split-bf16x3 tensor-core contractions, f32 projected problems) + f64 Rayleigh-Ritz",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if args.workload == BENCH_WORKLOAD else ws[0].name, "designs_per_step": 1, "k_per_design": w0.nk, "bands": w0.nbands,
                       "adjoint": "all-band weighted (every (k, band))",
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "roofline": roofline, "clocks": ck,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(st_mx.launches),
            "iterations": st_mx.iterations, "max_residual": st_mx.max_residual,
            "phase_ms_per_step": {"timed_in": "single-stream profiling pass",
                                  "block_iteration": st_pf.ms_iteration_loop / prof_steps,
                                  "iter_apply": st_pf.ms_iter_apply / prof_steps,
                                  "gram": st_pf.ms_gram / prof_steps,
                                  "update": st_pf.ms_update / prof_steps,
                                  "small_dense": st_pf.ms_small / prof_steps,
                                  "fp64_rayleigh_ritz": st_pf.ms_final_rr / prof_steps,
                                  "rr_gemm": st_pf.ms_rr_gemm / prof_steps,
                                  "adjoint": st_pf.ms_grad_kernels / prof_steps,
                                  "host_idle_between_iterations": st_pf.ms_host_idle / prof_steps,
                                  "last_set_design": st_pf.ms_setup, "last_bands": st_pf.ms_bands,
                                  "last_gap_and_grad": st_pf.ms_grad},
            "timed_run": {"k_halves_on_two_streams": True, "last_bands_ms": st_mx.ms_bands,
                          "last_set_design_ms": st_mx.ms_setup, "last_gap_and_grad_ms": st_mx.ms_grad},
            "roofline_families": fam,
            "fp64_form": fp64,
            "peaks_measured": {"fp64_tflops": fp64_peak / 1e3, "fp32_tflops": fp32_peak / 1e3}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == BENCH_WORKLOAD:
        line["cpu_baseline"] = cpu_baseline(args.cpu_k)
    if rank == 0:
        print(json.dumps(line), flush=True)
    s_mx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
