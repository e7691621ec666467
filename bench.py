"""Benchmark: time to the nev eigenpairs closest to exp(i phi) of the L = 20 kicked-Ising
Floquet operator (residual <= 1e-10), with the filter's U-application throughput against
the HBM roofline.

One step = one complete solve of the workload through the C ABI: operator set-up, the
Krylov-Schur Arnoldi on g_k(U) (filter sweeps, CGS2, small solve, restarts), Ritz vectors,
Rayleigh quotients and residuals, and (FILTER_FP32 form) the FP64 polish. Inputs are
synthetic: h_i ~ U[-1, 1] from a seeded generator, complex-Gaussian start vector.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 runs independent replicas (one disorder realisation per rank; no data-path
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
    if args.precision:
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
    prec = {"filter_fp32": floquet.FILTER_FP32, "fp64": floquet.FP64,
            "filter_df": floquet.FILTER_DF}[cfg["precision"]]
    d = 1 << L
    h = inputs.disorder(L, cfg["W"], replica_seed(cfg["seed"], rank))  # one per replica
    v0_host = inputs.start_vector(L)
    v0 = torch.from_numpy(v0_host).to(dev)
    evecs = torch.empty((nev, d), dtype=torch.complex128, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()

    def one_solve(v0_arg, evecs_arg):
        with floquet.Floquet(L, inputs.J_DEFAULT, inputs.G_DEFAULT, h) as fq:
            return fq.arnoldi_eigs(phi, k, nev, m, v0_arg, precision=prec,
                                   max_restarts=args.max_restarts, evecs=evecs_arg)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # Warm-up. The last warm-up step is the end-to-end measurement: the public C-ABI call
    # with HOST buffers (h and v0 in; eigenvalues, residuals and eigenvectors out), so the
    # host<->device copies are inside its timed region.
    evecs_host = np.empty((nev, d), dtype=np.complex128)
    t_e2e, e2e_res = None, None
    for w in range(args.warmup):
        flush.fill_(1.0)
        barrier()
        if w == args.warmup - 1:
            te = time.perf_counter()
            e2e_res = one_solve(v0_host, evecs_host)
            barrier()
            t_e2e = time.perf_counter() - te
        else:
            one_solve(v0, evecs)

    sampler = ClockSampler(local)
    sampler.start()
    floquet.profile_enable(True)
    floquet.reset_launch_count()
    times = []
    results = None
    for _ in range(args.steps):
        flush.fill_(1.0)
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        results = one_solve(v0, evecs)
        t1.record(stream)
        barrier()
        times.append(t0.elapsed_time(t1) / 1000.0)
    launches = floquet.launch_count()
    prof = floquet.profile_read()
    floquet.profile_enable(False)
    clocks = sampler.stop()

    t_step = max_over_ranks(sum(times) / len(times), dev)
    if t_e2e is None:  # no warm-up: measure the end-to-end call now
        barrier()
        te = time.perf_counter()
        e2e_res = one_solve(v0_host, evecs_host)
        barrier()
        t_e2e = time.perf_counter() - te
    om_e, res_e, nconv_e, rc_e = e2e_res

    om, res, nconv, rc = results
    kind = {floquet.FILTER_FP32: "c64", floquet.FP64: "c128", floquet.FILTER_DF: "df"}[prec]
    sweep_ms, u_apps, alg_bytes = prof[kind]
    hbm, peak_kind = _peaks()
    form = os.environ.get("FLOQUET_KRYLOV_FORM", "horner")
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
            ipa = df_instr_per_amplitude(L, form)
            ach_t = ipa * d * u_apps / (sweep_ms / 1e3) / 1e12
            roofline = {"bound": "alu", "achieved": round(ach_t, 2), "peak": round(peak_t, 2),
                        "unit": "T FP32 instr/s", "frac": round(ach_t / peak_t, 4),
                        "traffic": traffic, "kernel": "U application (pass_pipe_kernel x2)",
                        "fp32_instr_per_amplitude": ipa, "u_applications": int(u_apps),
                        "sweep_s": round(sweep_ms / 1e3, 3),
                        "peak_source": f"derived: {N_SM} SMs x {FP32_LANES} FP32 lanes x "
                                       f"{mhz:.0f} MHz (MEASURED_PEAKS.json sm_max_mhz)",
                        "hbm_view": hbm_view}
        else:
            roofline = dict(hbm_view, kernel="U application (pass kernels)",
                            u_applications=int(u_apps), sweep_s=round(sweep_ms / 1e3, 3))
        out = {
            "metric": METRIC, "value": round(t_step, 4), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_step * 1e3, 2),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": {"c64": "c64 sweeps / f64 Arnoldi", "c128": "c128 / f64",
                      "df": "double-float (2 x f32) sweeps / f64 Arnoldi"}[kind],
            "data": "synthetic (seeded h_i ~ U[-1,1], complex-Gaussian start vector)",
            "config": {"workload": args.workload, "L": L, "J": inputs.J_DEFAULT,
                       "g": inputs.G_DEFAULT, "W": cfg["W"], "phi": phi, "k": k, "m": m,
                       "nev": nev, "precision": cfg["precision"],
                       "filter_form": os.environ.get("FLOQUET_KRYLOV_FORM", "horner"),
                       "parallelism": f"replicas x{ws}",
                       "l2": "working set larger than L2 (Krylov basis 4 GiB) and a 256 MiB "
                             "buffer written between steps"},
            "result": {"status": rc, "n_conv": nconv, "max_resid": float(np.max(res)),
                       "omega_first": [float(om[0].real), float(om[0].imag)]},
            "e2e": {"value": round(t_e2e, 4), "unit": UNIT,
                    "h2d_bytes_per_step": int(d * 16 + L * 8),
                    "d2h_bytes_per_step": int(nev * d * 16 + nev * 24),
                    "status": rc_e, "n_conv": nconv_e},
            "roofline": roofline,
            "gpu_launches": int(launches // max(1, args.steps)),
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(cfg, u_apps // max(1, args.steps), h,
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
    name = "pass_pipe_kernel" if kind == "df" else "pass_kernel"
    p = os.path.join(ROOT, "profiles", f"{name}_L{L}_{kind}_traffic.json")
    if kind in _CURRENT_TRAFFIC and os.path.exists(p):
        with open(p) as f:
            return json.load(f).get("dram_bytes_per_u_application")
    return None


def cpu_baseline(cfg, u_apps_per_solve, h, seconds=15.0):
    """The oracle as it stands on the host cores: time oracle U applications at the
    workload's L for ~`seconds`, then scale to the U applications one GPU solve performed
    (the filter sweeps dominate the solve; CGS2 and the small solves are not counted, so the
    CPU figure is a lower bound)."""
    from oracle import model

    from paper_2102_05054_gb300 import inputs
    L = cfg["L"]
    op = model.KickedIsing(L, inputs.J_DEFAULT, inputs.G_DEFAULT, h)
    psi = inputs.complex_gaussian(1 << L, 1)
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds or n < 2:
        psi = op.apply_u(psi)
        n += 1
    dt = (time.perf_counter() - t0) / n
    total = dt * u_apps_per_solve
    return {"value": round(total, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} oracle U applications at L={L} ({dt:.3f} s each, numpy, one "
                      f"thread) scaled to the {u_apps_per_solve} U applications of one GPU "
                      f"solve; host has {os.cpu_count()} cores"}


def run_reference(args):
    """--impl reference: the CPU oracle on this machine's host cores, bounded sample per step."""
    from oracle import model

    from paper_2102_05054_gb300 import inputs
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    cfg = _cfg(args)
    L, k, m = cfg["L"], cfg["k"], cfg["m"]
    h = inputs.disorder(L, cfg["W"], cfg["seed"])
    op = model.KickedIsing(L, inputs.J_DEFAULT, inputs.G_DEFAULT, h)
    # U applications of one solve: at least m filters of k - 1 applications (one Krylov build)
    u_apps = m * (k - 1)
    psi = inputs.complex_gaussian(1 << L, 1)
    vals = []
    for step in range(args.warmup + args.steps):
        n = 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < args.ref_seconds or n < 1:
            psi = op.apply_u(psi)
            n += 1
        if step >= args.warmup:
            vals.append((time.perf_counter() - t0) / n * u_apps)
    v = sum(vals) / len(vals)
    out = {"metric": METRIC, "value": round(v, 1), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v * 1e3, 1),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded h_i ~ U[-1,1])", "impl": "reference",
           "config": {"workload": args.workload, "L": L, "k": k, "m": m, "nev": cfg["nev"],
                      "parallelism": "host cores"},
           "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"oracle U applications for ~{args.ref_seconds} s per "
                                      f"step, scaled to m*(k-1) = {u_apps} applications "
                                      f"(one Krylov build); host has {os.cpu_count()} cores"},
           "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="filter_df",
                    choices=["fp64", "filter_fp32", "filter_df"])
    ap.add_argument("--max-restarts", type=int, default=30)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
