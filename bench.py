"""Benchmark: time to the nev eigenpairs closest to exp(i phi) of the L = 20 kicked-Ising
Floquet operator (every residual <= 1e-10), with the filter's U-application throughput
against its roofline.

One step = one eigenproblem of the workload: a disorder realisation of its own (h_i ~ U[-1, 1],
seeded), solved through the C ABI from the start vector to the nev pairs -- operator set-up,
the Krylov-Schur Arnoldi on g_k(U) (filter sweeps, CGS2, small solves), Ritz vectors,
Rayleigh quotients and FP64 residuals. Steps run --batch at a time in one lockstep solve
(arnoldi_eigs_batched: the filter sweeps of the batch share each launch), so `value` is the
solve time per eigenproblem at that batch size; a single problem's latency is the batch's
solve time (reported as `latency_s`). Inputs are synthetic.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 runs independent replicas (realisations of their own per rank; no data-path
collective), launched with torch.distributed.run.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "L=20 time to nev eigenpairs (resid<=1e-10); U-apply GB/s vs HBM peak"
UNIT = "s"
WORKLOAD = "kicked_ising_L20"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# FP32 pipe: 152 SMs x 128 lanes, one FP32 instruction (FADD, FMUL or FFMA) per lane per clock
N_SM, FP32_LANES = 152, 128


def _fp32_peak_tops():
    """FP32 instructions per second at the maximum SM clock (units x clock)."""
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return N_SM * FP32_LANES * mhz * 1e6 / 1e12, mhz


def df_instr_per_amplitude(L, form):
    """Algorithmic FP32 instructions per amplitude of one double-float U application: each
    kicked qubit gives two real outputs per amplitude, each an error-free x + tau*y (12 FP32
    instructions: exact product 2, two-sum 6, low-order terms 4); the epilogue is one
    double-float complex product for the phase (44) and, for the Horner form, one complex
    multiply-add (60) or, for the accumulate form, a second product plus the multiply-add
    (104)."""
    return 24 * L + (104 if form == "horner" else 148)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(base_seed, rank):
    """Disorder seed of the realisation a replica solves: independent problems per rank
    (weak scaling, no data-path collective)."""
    return base_seed + rank


def step_seeds(base_seed, rank, steps):
    """Disorder seeds of the K steps of one rank: realisation i of rank r uses
    replica_seed(base_seed, r * K + i), so no two steps or ranks solve the same problem."""
    return [replica_seed(base_seed, rank * steps + i) for i in range(steps)]


def batches(steps, batch):
    """Sizes of the lockstep solves that cover `steps` problems, `batch` at a time."""
    out = []
    left = steps
    while left > 0:
        out.append(min(batch, left))
        left -= out[-1]
    return out


def max_over_ranks(value, device):
    """Max of a per-rank float over the process group (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _cfg(args):
    from paper_2102_05054_gb300 import inputs
    c = dict(inputs.WORKLOADS[args.workload])
    c["precision"] = args.precision
    return c


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2102_05054_gb300 import floquet, inputs

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = _cfg(args)
    L, k, m, nev, phi = cfg["L"], cfg["k"], cfg["m"], cfg["nev"], cfg["phi"]
    prec = {"fp64": floquet.FP64, "filter_df": floquet.FILTER_DF}[cfg["precision"]]
    d = 1 << L
    seeds = step_seeds(cfg["seed"], rank, args.steps)
    hs = np.stack([inputs.disorder(L, cfg["W"], s) for s in seeds])  # one realisation per step
    v0_pinned = torch.from_numpy(inputs.start_vector(L)).pin_memory()
    v0 = torch.empty(d, dtype=torch.complex128, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()
    phis = np.array([phi])

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # Warm-up: no solves. Each warm-up builds an operator of the workload and runs a short
    # filter with the batch width and sweep precision of the timed solves (module load, kernel
    # images, the launch-shape autotuner's code paths, CUDA graph machinery).
    sweep = {floquet.FP64: floquet.C128, floquet.FILTER_DF: floquet.C128_DF}[prec]
    nb0 = batches(args.steps, args.batch)[0] if args.steps > 0 else args.batch
    for w in range(args.warmup):
        with floquet.Floquet(L, inputs.J_DEFAULT, inputs.G_DEFAULT, hs[0]) as fq:
            x = torch.zeros((nb0, d), dtype=torch.complex128, device=dev)
            x[:, 0] = 1.0
            y = torch.empty_like(x)
            fq.filter_apply(phi, 9, x, y, form=floquet.FORM_HORNER, sweep=sweep)
        barrier()

    sampler = ClockSampler(local)
    sampler.start()
    floquet.profile_enable(True)
    floquet.reset_launch_count()
    dev_s, wall_s, lat = [], [], []
    results = []
    i0 = 0
    for nb in batches(args.steps, args.batch):
        hb = hs[i0:i0 + nb]
        flush.fill_(1.0)
        barrier()
        # e2e: the step's inputs from pinned host memory, the public C-ABI call, results on the
        # host; value: the device time of the same call, inputs already resident
        t0 = time.perf_counter()
        v0.copy_(v0_pinned, non_blocking=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        om, res, nconv, rc = floquet.arnoldi_eigs_batched(
            L, inputs.J_DEFAULT, inputs.G_DEFAULT, hb, phis, k, nev, m, v0,
            tol=args.tol, precision=prec, max_restarts=args.max_restarts)
        e1.record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        dev_s.append(e0.elapsed_time(e1) / 1000.0)
        wall_s.append(t1 - t0)
        lat.append(dev_s[-1])
        results.append((om, res, nconv, rc, nb))
        i0 += nb
    launches = floquet.launch_count()
    prof = floquet.profile_read()
    floquet.profile_enable(False)
    clocks = sampler.stop()

    t_step = max_over_ranks(sum(dev_s) / args.steps, dev)
    t_e2e = max_over_ranks(sum(wall_s) / args.steps, dev)
    kind = {floquet.FP64: "c128", floquet.FILTER_DF: "df"}[prec]
    sweep_ms, u_apps, alg_bytes = prof[kind]
    max_res = max(float(np.max(r[1])) for r in results)
    n_conv = int(sum(int(np.sum(r[2])) for r in results))
    status = [int(r[3]) for r in results]
    hbm, peak_kind = _peaks()
    out = None
    if rank == 0:
        achieved = alg_bytes / (sweep_ms / 1e3) / 1e9 if sweep_ms > 0 else None
        traffic = _ncu_traffic(L, kind)
        hbm_view = {"bound": "hbm", "achieved": round(achieved, 1) if achieved else None,
                    "peak": hbm, "unit": "GB/s",
                    "frac": round(achieved / hbm, 4) if achieved else None,
                    "traffic": traffic,
                    "bytes_per_u_application": int(round(alg_bytes / u_apps)) if u_apps
                    else None,
                    "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"}
        if kind == "df" and sweep_ms > 0:
            # the double-float sweep is bound by the FP32 pipe: algorithmic FP32 instructions
            # per U application against the FP32 issue rate at the maximum clock
            peak_t, mhz = _fp32_peak_tops()
            ipa = df_instr_per_amplitude(L, "horner")
            ach_t = ipa * d * u_apps / (sweep_ms / 1e3) / 1e12
            roofline = {"bound": "alu", "achieved": round(ach_t, 2), "peak": round(peak_t, 2),
                        "unit": "T FP32 instr/s", "frac": round(ach_t / peak_t, 4),
                        "traffic": traffic,
                        "kernel": "U application (double-float pass kernels, Horner filter)",
                        "fp32_instr_per_amplitude": ipa, "u_applications": int(u_apps),
                        "sweep_s": round(sweep_ms / 1e3, 3),
                        "peak_source": f"derived: {N_SM} SMs x {FP32_LANES} FP32 lanes x "
                                       f"{mhz:.0f} MHz (MEASURED_PEAKS.json sm_max_mhz)",
                        "hbm_view": hbm_view}
        else:
            roofline = dict(hbm_view, kernel="U application (Horner filter)",
                            u_applications=int(u_apps), sweep_s=round(sweep_ms / 1e3, 3))
        h2d = int(d * 16 + L * 8)  # start vector and the step's field h, per step
        d2h = int(nev * 24 + 4)   # eigenvalues, residuals and n_conv, per step
        out = {
            "metric": METRIC, "value": round(t_step, 4), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_step * 1e3, 2),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": {"df": "double-float (2 x f32) sweeps / f64 Arnoldi",
                      "c128": "c128 sweeps / f64 Arnoldi"}[kind],
            "data": "synthetic (seeded h_i ~ U[-1,1], one realisation per step; complex-"
                    "Gaussian start vector)",
            "config": {"workload": args.workload, "L": L, "J": inputs.J_DEFAULT,
                       "g": inputs.G_DEFAULT, "W": cfg["W"], "phi": phi, "k": k, "m": m,
                       "nev": nev, "precision": cfg["precision"], "filter_form": "horner",
                       "batch": args.batch, "krylov_tol": args.tol,
                       "parallelism": f"replicas x{ws}",
                       "l2": "working set larger than L2 (Krylov bases 4 GiB per problem) and "
                             "a 256 MiB buffer written before every batch"},
            "latency_s": round(max(lat), 3),
            "result": {"status": status, "n_conv": n_conv, "problems": args.steps,
                       "max_resid": max_res},
            "e2e": {"value": round(t_e2e, 4), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": roofline,
            "gpu_launches": int(launches // max(1, args.steps)),
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(cfg, u_apps // max(1, args.steps), hs[0],
                                               seconds=args.cpu_seconds)
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


# Kernels whose committed ncu counters were taken on the current code (others report null).
_CURRENT_TRAFFIC = {"df"}


def _ncu_traffic(L, kind):
    """DRAM bytes per U application from the committed ncu summary, if one matches the
    current kernel."""
    p = os.path.join(ROOT, "profiles", f"pass_pipe_kernel_L{L}_{kind}_traffic.json")
    if kind in _CURRENT_TRAFFIC and os.path.exists(p):
        with open(p) as f:
            return json.load(f).get("dram_bytes_per_u_application")
    return None


def _oracle_worker(args):
    """One host process: oracle U applications at L for about `seconds` (numpy, one BLAS
    thread); returns (applications, elapsed)."""
    L, h, seconds, seed = args
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import model

    from paper_2102_05054_gb300 import inputs
    op = model.KickedIsing(L, inputs.J_DEFAULT, inputs.G_DEFAULT, h)
    psi = inputs.complex_gaussian(1 << L, seed)
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds or n < 1:
        psi = op.apply_u(psi)
        n += 1
    return n, time.perf_counter() - t0


def oracle_throughput(L, h, seconds, workers):
    """U applications per second of the oracle on `workers` host processes, each applying U
    to an independent vector (a spawn pool: safe after the GPU is in use)."""
    import multiprocessing as mp
    if workers <= 1:
        n, dt = _oracle_worker((L, h, seconds, 7))
        return n / dt, 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_worker, [(L, h, seconds, 7 + i) for i in range(workers)])
    return sum(n / dt for n, dt in res), workers


def cpu_baseline(cfg, u_apps_per_solve, h, seconds=10.0):
    """The oracle as it stands on the host cores: oracle U applications at the workload's L,
    one process per core on independent vectors for ~`seconds`, projected to the U
    applications of one GPU solve (the filter sweeps dominate the solve; CGS2 and the small
    solves are not counted, so the CPU figure is a lower bound)."""
    L = cfg["L"]
    workers = os.cpu_count() or 1
    rate, used = oracle_throughput(L, h, seconds, workers)
    total = u_apps_per_solve / rate
    return {"value": round(total, 1), "unit": UNIT, "cores": used, "kind": "oracle",
            "projected": True,
            "sample": f"oracle U applications at L={L} (numpy, {used} processes x 1 BLAS "
                      f"thread, ~{seconds:.0f} s each): {rate:.2f} applications/s in total, "
                      f"projected to the {u_apps_per_solve} U applications of one GPU solve; "
                      f"host has {os.cpu_count()} cores"}


def run_reference(args):
    """--impl reference: the CPU oracle on this machine's host cores, bounded sample per step,
    projected to one solve."""
    from paper_2102_05054_gb300 import inputs
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    cfg = _cfg(args)
    L, k, m = cfg["L"], cfg["k"], cfg["m"]
    h = inputs.disorder(L, cfg["W"], cfg["seed"])
    # U applications of one solve: at least m filters of k - 1 applications (one Krylov build)
    u_apps = m * (k - 1)
    workers = os.cpu_count() or 1
    vals = []
    for step in range(args.warmup + args.steps):
        rate, used = oracle_throughput(L, h, args.ref_seconds, workers)
        if step >= args.warmup:
            vals.append(u_apps / rate)
    v = sum(vals) / len(vals)
    sample = (f"oracle U applications for ~{args.ref_seconds} s per step on {used} host "
              f"processes (one BLAS thread each), projected to m*(k-1) = {u_apps} "
              f"applications (one Krylov build); host has {os.cpu_count()} cores")
    out = {"metric": METRIC, "value": round(v, 1), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v * 1e3, 1),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded h_i ~ U[-1,1])", "impl": "reference",
           "config": {"workload": args.workload, "L": L, "k": k, "m": m, "nev": cfg["nev"],
                      "parallelism": "host cores"},
           "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": used, "kind": "oracle",
                            "projected": True, "sample": sample},
           "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def u_timing(Ls, nvecs=(1, 2, 4), k=513, reps=3):
    """Per-U-application time of the Horner filter (k terms, CUDA events on the launching
    stream, after two warm-up filters) for each sweep precision, state count and L: one JSON
    line per case. The filter runs whatever launch shape the autotuner picked for the
    operator (FLOQUET_VERBOSE=1 prints the tuner's timings)."""
    import torch

    from paper_2102_05054_gb300 import floquet, inputs
    names = {floquet.C64: "c64", floquet.C128_DF: "df", floquet.C128: "c128"}
    for L in Ls:
        d = 1 << L
        h = inputs.disorder(L, 1.0, 1)
        for sweep in (floquet.C64, floquet.C128_DF, floquet.C128):
            for nvec in nvecs:
                if sweep == floquet.C128 and nvec > 1:
                    continue
                dt = torch.complex64 if sweep == floquet.C64 else torch.complex128
                with floquet.Floquet(L, inputs.J_DEFAULT, inputs.G_DEFAULT, h) as fq:
                    x = torch.from_numpy(inputs.random_states(d, nvec, 3).T.copy()).to(dt).cuda()
                    y = torch.empty_like(x)
                    stream = torch.cuda.current_stream()
                    for _ in range(2):
                        fq.filter_apply(0.0, k, x, y, form=floquet.FORM_HORNER, sweep=sweep)
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(reps):
                        fq.filter_apply(0.0, k, x, y, form=floquet.FORM_HORNER, sweep=sweep)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    us = 1000.0 * e0.elapsed_time(e1) / (reps * (k - 1) * nvec)
                b = 8 if sweep == floquet.C64 else 16
                print(json.dumps({"L": L, "sweep": names[sweep], "nvec": nvec, "k": k,
                                  "us_per_u_application": round(us, 3),
                                  "horner_bytes_per_u": 3 * d * b,
                                  "gbs_algorithmic": round(3 * d * b / us / 1e3, 1)}),
                      flush=True)


def km_grid(L, nev, k0, m0, max_m=512):
    """(k, m) points of the parameter scan (the paper's Fig. bench scans the filter length and
    the Krylov dimension): k in k0 x {1/4, 1/2, 1, 2} (at least 2, at most d / 2) and m in
    m0 x {0.75, 1, 1.5, 2} (at least nev + 16, the room a convergence check needs, at most
    min(max_m, d - 1)); duplicates removed, sorted."""
    d = 1 << L
    ks = sorted({int(min(max(2, round(k0 * f)), d // 2)) for f in (0.25, 0.5, 1.0, 2.0)})
    ms = sorted({int(min(max(nev + 16, round(m0 * f)), max_m, d - 1))
                 for f in (0.75, 1.0, 1.5, 2.0)})
    return [(k, m) for k in ks for m in ms if m > nev]


def km_scan(args):
    """Time to the workload's nev pairs (every residual <= 1e-10) for each (k, m) of
    km_grid around the workload's own pair, plus the paper's rule (suggest_params): one JSON
    line per point (CUDA events around one solve; U applications from the library's
    profiling hook), then the fastest point."""
    import torch

    from paper_2102_05054_gb300 import floquet, inputs
    cfg = _cfg(args)
    L, nev, phi = cfg["L"], cfg["nev"], cfg["phi"]
    prec = {"fp64": floquet.FP64, "filter_df": floquet.FILTER_DF}[cfg["precision"]]
    kind = {floquet.FP64: "c128", floquet.FILTER_DF: "df"}[prec]
    pts = km_grid(L, nev, cfg["k"], cfg["m"])
    rule = floquet.suggest_params(L, nev)
    if rule not in pts:
        pts.append(rule)
    h = inputs.disorder(L, cfg["W"], cfg["seed"])
    v0 = torch.from_numpy(inputs.start_vector(L)).cuda()
    stream = torch.cuda.current_stream()
    best = None
    for (k, m) in pts:
        with floquet.Floquet(L, inputs.J_DEFAULT, inputs.G_DEFAULT, h) as fq:
            floquet.profile_enable(True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            om, res, nconv, rc = fq.arnoldi_eigs(phi, k, nev, m, v0, tol=args.tol,
                                                 precision=prec,
                                                 max_restarts=args.max_restarts, check=False)
            e1.record(stream)
            torch.cuda.synchronize()
            prof = floquet.profile_read()
            floquet.profile_enable(False)
        t = e0.elapsed_time(e1) / 1000.0
        ok = rc == floquet.OK and nconv == nev and float(np.max(res)) <= 1e-10
        line = {"L": L, "nev": nev, "k": k, "m": m, "paper_rule": (k, m) == rule,
                "seconds": round(t, 3), "status": int(rc), "n_conv": int(nconv),
                "max_resid": float(np.max(res)) if len(res) else None,
                "u_applications": int(prof[kind][1]), "precision": cfg["precision"]}
        print(json.dumps(line), flush=True)
        if ok and (best is None or t < best["seconds"]):
            best = line
    print(json.dumps({"fastest": best, "paper_rule": list(rule)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="filter_df", choices=["fp64", "filter_df"])
    ap.add_argument("--batch", type=int, default=2,
                    help="eigenproblems per lockstep solve")
    ap.add_argument("--tol", type=float, default=1e-6,
                    help="Krylov convergence tolerance of the Ritz values of g_k (the U-residual "
                         "<= 1e-10 of every returned pair is checked separately)")
    ap.add_argument("--max-restarts", type=int, default=30)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=5.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--km-scan", action="store_true",
                    help="time the workload's solve over a (k, m) grid around its own pair and "
                         "the paper's rule instead of the benchmark line")
    ap.add_argument("--u-timing", default=None,
                    help="comma-separated L values: print per-U-application filter times per "
                         "sweep precision instead of the benchmark line")
    args = ap.parse_args()
    if args.u_timing:
        u_timing([int(x) for x in args.u_timing.split(",")])
        return
    if args.km_scan:
        km_scan(args)
        return
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
