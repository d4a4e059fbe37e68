"""Benchmark of the master-equation hot path: QME steps/s (and complex TFLOP/s).

One bench step = one complete evolution of the hydrogen-bond-shaped workload (dim 512,
10000 QME steps of dt = 0.05, populations every 100 steps) through qed_evolve, with rho
resident in HBM.  The library's split-precision path is timed; the all-FP64 GPU path is
timed beside it on a shorter run, and the FP64 CPU oracle on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision split_fp16x2|fp64] [--qme-steps S]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank evolves its own replica
of the workload: replicas only, no collective on the data path.
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

import qed_workloads as W  # noqa: E402

WORKLOAD = "hb_shaped_d512"
METRIC = "QME steps/s (split-precision, complex TFLOP/s alongside) at max|drho|<=1e-5 vs oracle"
L2_FLUSH_BYTES = 512 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="split_fp16x2")
    p.add_argument("--autotune", action="store_true", help="time the tile choices before the run (qed_autotune)")
    p.add_argument("--scheme", default="lie", choices=["lie", "strang"],
                   help="time-stepping scheme (the adjoint workload differentiates the Lie step only)")
    p.add_argument("--qme-steps", type=int, default=None)
    p.add_argument("--fp64-qme-steps", type=int, default=200)
    p.add_argument("--cpu-sample", type=int, default=40, help="oracle QME steps in the CPU baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default=WORKLOAD,
                   choices=[WORKLOAD, "jch2_d36", "lattice_32x32_d2049", "batched_chains",
                            "adjoint_lattice_24x24_d1153", "selection_hb_shaped_d512", "photon_plane_81x51_d4131",
                            "hb_two_bonds_d4096"],
                   help="the default is the headline workload; the others are measured with --workload")
    p.add_argument("--instances", type=int, default=512, help="batched_chains: number of instances")
    p.add_argument("--selection-eps", type=float, default=1e-20, help="selection workload: threshold")
    p.add_argument("--selection-round", type=int, default=100, help="selection workload: steps per round")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms, world, device):
    """The slowest replica's time (ms): the whole job finishes when its slowest rank does."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms):
    """Units per second of all replicas together (each rank runs units_per_rank)."""
    return world * units_per_rank / (ms / 1e3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def oracle_rate(model, n_steps):
    """The FP64 CPU oracle, as it stands, on n_steps of the workload: QME steps/s."""
    import oracle
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] or [os.cpu_count()])
    except Exception:
        cores = os.cpu_count()
    basis = oracle.enumerate_basis(model)
    H = oracle.hamiltonian(model, basis)
    U = oracle.propagator(H, model["dt"])
    jumps = oracle.jump_operators(model, basis)
    rho = oracle.initial_density(model, basis)
    t0 = time.perf_counter()
    for _ in range(n_steps):
        rho = oracle.step(rho, U, jumps, model["dt"])
    dt = time.perf_counter() - t0
    return n_steps / dt, cores, dt


def complex_tflops(D, steps_per_s):
    return 16.0 * D ** 3 * steps_per_s / 1e12


def run_reference(args):
    world, rank, _ = dist_env()
    if world > 1 and rank != 0:
        return
    model = W.hb_shaped()
    D = 512
    sample = max(1, args.cpu_sample // 2)
    for _ in range(args.warmup):
        oracle_rate(model, 2)
    total_t, total_n, cores = 0.0, 0, os.cpu_count()
    for _ in range(args.steps):
        rate, cores, dt = oracle_rate(model, sample)
        total_t += dt
        total_n += sample
    value = total_n / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "QME steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "dim": D, "qme_steps_per_step": 10000,
                                        "dt": 0.05, "record_every": 100, "precision": "fp64 (CPU oracle)",
                                        "sample_qme_steps_per_step": sample},
        "complex_tflops": complex_tflops(D, value),
        "cpu_baseline": {"value": value, "unit": "QME steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} QME steps of the dim-512 workload per bench step"},
        "e2e": {"value": value, "unit": "QME steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2403_07042_gb300 as qed
    from paper_2403_07042_gb300 import build as qbuild

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    qbuild.build()

    model = W.hb_shaped()
    qme_steps = args.qme_steps or model["n_steps"]
    r = model["record_every"]
    gm = qed.Model(model, precision=args.precision, scheme=args.scheme)
    tuned = gm.autotune(20) if args.autotune else None
    D = gm.dim
    obs = list(range(D))
    i0 = gm.initial_index()
    rho0 = torch.zeros((D, D), dtype=torch.complex128, device=dev)
    rho0[i0, i0] = 1.0
    rho = rho0.clone()
    n_rec = gm.n_records(qme_steps, r)
    records = torch.zeros((n_rec, len(obs)), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def one_step():
        rho.copy_(rho0)
        gm.evolve(rho, qme_steps, record_every=r, obs_ids=obs, records=records)

    for _ in range(args.warmup):
        one_step()
    gm.sync()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    launches0 = qed.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))          # L2 flush between timed iterations (outside the events)
        ev[k][0].record(stream)
        one_step()
        ev[k][1].record(stream)
    barrier()
    launches = qed.launch_count() - launches0
    clocks = sampler.stop()
    gm.sync()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    t_max = max_over_ranks(t_ms, world, dev)
    value = whole_job_rate(world, args.steps * qme_steps, t_max)

    # parity of this run's final state against the stored oracle trajectory, if present
    parity = parity_against_golden(rho, records, qme_steps) if args.scheme == "lie" else None

    # end to end: pinned host rho0 -> device, evolve, records + final rho -> host
    h_rho0 = rho0.cpu().pin_memory()
    h_rho = torch.empty_like(h_rho0).pin_memory()
    h_rec = torch.empty(records.shape, dtype=records.dtype).pin_memory()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for k in range(args.steps):
        flush.fill_(float(k))
        e0.record(stream)
        rho.copy_(h_rho0, non_blocking=True)
        gm.evolve(rho, qme_steps, record_every=r, obs_ids=obs, records=records)
        h_rec.copy_(records, non_blocking=True)
        h_rho.copy_(rho, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e_value = whole_job_rate(world, args.steps * qme_steps, e2e_ms)

    # kernel classes timed live with CUDA events on the launching stream
    prof_steps = min(500, qme_steps)
    rho.copy_(rho0)
    kern = gm.profile(rho, prof_steps)
    roofline = make_roofline(kern, D, args.precision)
    roofline_dissipator = dissipator_roofline(kern, D)

    # the all-FP64 GPU path on the same workload (shorter run)
    fp64 = None
    if args.precision != "fp64" and args.fp64_qme_steps > 0:
        g64 = qed.Model(model, precision="fp64", scheme=args.scheme)
        rho64 = rho0.clone()
        g64.evolve(rho64, 5)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g64.evolve(rho64, args.fp64_qme_steps)
        b.record(stream)
        b.synchronize()
        rate64 = args.fp64_qme_steps / (a.elapsed_time(b) / 1e3)
        fp64 = {"steps_per_s": rate64, "complex_tflops": complex_tflops(D, rate64),
                "qme_steps_timed": args.fp64_qme_steps, "speedup_split_over_fp64": value / world / rate64}
        g64.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, cores, _ = oracle_rate(model, args.cpu_sample)
        cpu = {"value": rate, "unit": "QME steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample} QME steps of the dim-512 workload (full run: {qme_steps})"}
    step_bytes_in = rho0.numel() * 16
    step_bytes_out = records.numel() * 8 + rho.numel() * 16
    line = {
        "metric": METRIC, "value": value, "unit": "QME steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16x2->f32 (split), f64 master" if args.precision != "fp64" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "dim": D, "qme_steps_per_step": qme_steps, "dt": model["dt"],
                   "record_every": r, "precision": args.precision, "scheme": args.scheme, "autotuned": tuned,
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed (512 MB write) between timed iterations; working set < L2 within a run"},
        "complex_tflops": complex_tflops(D, value / world) * world,
        "parity_vs_oracle": parity,
        "fp64_gpu": fp64,
        "roofline": roofline,
        "roofline_dissipator": roofline_dissipator,
        "kernels_ms_per_qme_step": kern,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "QME steps/s", "h2d_bytes_per_step": step_bytes_in,
                "d2h_bytes_per_step": step_bytes_out},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def dissipator_roofline(kern, D):
    """The Lindblad update's achieved bandwidth against the measured HBM copy rate: the
    algorithmic bytes are the element's V read (16 B), the new rho written (16 B) and its
    FP16 planes written (8 B), per complex element (the gathers of the jump terms come on
    top).  Its operands sit in L2 at these sizes, so the fraction is a lower bound of what the
    memory system delivers."""
    name = "dissipate" if "dissipate" in kern else ("dissipate_f64" if "dissipate_f64" in kern else None)
    if not name or kern[name] <= 0:
        return None
    peaks, src = measured_peaks()
    achieved = 40.0 * D * D / (kern[name] * 1e-3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "bytes_per_element": 40, "peak_source": src}


# dram__bytes_read.sum + dram__bytes_write.sum of one GEMM1 launch (ncu, warm L2)
GEMM1_DRAM_BYTES_D512 = 256


def make_roofline(kern, D, precision):
    peaks, src = measured_peaks()
    if not kern:
        return None
    name, ms = max(kern.items(), key=lambda kv: kv[1])
    if precision == "fp64":
        # complex FP64 GEMM: 8 D^3 flop per product on the FP64 pipes
        flops = 8.0 * D ** 3
        peak = 1.25e3 * peaks.get("sm_max_mhz", 2070.0) / 2070.0  # GFLOP/s nominal at max clock
        achieved = flops / (ms * 1e-3) / 1e9
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                "frac": achieved / peak, "traffic": None, "peak_source": "nominal FP64 1.25 TFLOP/s"}
    if name.startswith("gemm"):
        # executed MMA work over the real embedding, padded Dp: GEMM1 (2Dp x Dp x 2Dp) with
        # four FP16 plane products, GEMM2 (Dp x 2Dp x 2Dp) with three
        Dp = -(-D // 128) * 128
        segs = 4 if name.startswith("gemm1") else 3
        flops = 2.0 * (2 * Dp) * Dp * (2 * Dp) * segs
        achieved = flops / (ms * 1e-3) / 1e12
        peak = peaks["bf16_tflops"]
        # DRAM bytes per launch from one ncu capture of this kernel in the steady state of the
        # dim-512 step (profiles/tc_gemm_hb_shaped_d512_full.md): the operands stay in L2
        traffic = GEMM1_DRAM_BYTES_D512 if (name.startswith("gemm1") and D == 512) else None
        return {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": f"{src} bf16 dense burst (fp16 has the same nominal rate)"}
    # element-wise update: bytes per element
    bytes_ = 56.0 * D * D
    achieved = bytes_ / (ms * 1e-3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": src}


def parity_against_golden(rho, records, qme_steps):
    path = os.path.join(ROOT, "tests", "golden", "hb_shaped_d512_oracle.npz")
    if not os.path.exists(path) or qme_steps != 10000:
        return None
    g = np.load(path)
    pop = records.cpu().numpy()
    rho_h = rho.cpu().numpy()
    out = {"max_abs_pop": float(np.abs(pop - g["records"]).max())}
    if "rho_rows" in g:
        rows = g["rho_rows"]
        out["max_abs_rho_sampled_rows"] = float(np.abs(rho_h[rows] - g["rho_sample"]).max())
    return out


def run_other(args):
    """Secondary workloads (one GPU, no collectives): the dim-36 FP64 cavities, the 32 x 32
    lattice, the batched chains and the adjoint lattice.  Same JSON fields; `config.workload`
    names the workload."""
    import torch

    import paper_2403_07042_gb300 as qed
    from paper_2403_07042_gb300 import build as qbuild

    qbuild.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    wl = args.workload
    prec = args.precision
    extra = {}
    if wl == "batched_chains":
        specs = W.batched_chains(args.instances, seed=0)
        steps = args.qme_steps or specs[0]["n_steps"]
        models = [qed.Model(m, precision=prec, scheme=args.scheme) for m in specs]
        dims = [gm.dim for gm in models]
        rho0 = []
        for gm in models:
            r = torch.zeros((gm.dim, gm.dim), dtype=torch.complex128, device=dev)
            i0 = gm.initial_index()
            r[i0, i0] = 1.0
            rho0.append(r)
        rhos = [r.clone() for r in rho0]

        def one():
            for a, b in zip(rhos, rho0):
                a.copy_(b)
            qed.evolve_batched(models, rhos, steps)
        flops = sum(16.0 * d ** 3 for d in dims)
        unit = "instance QME steps/s"
        per_step_units = len(models) * steps
        extra["dims"] = {"min": min(dims), "max": max(dims), "mean": float(np.mean(dims)),
                         "hist_128": np.histogram(dims, bins=range(0, 1153, 128))[0].tolist()}
    else:
        m = {"jch2_d36": W.jch_two_cavities, "lattice_32x32_d2049": W.lattice,
             "adjoint_lattice_24x24_d1153": W.adjoint_lattice, "selection_hb_shaped_d512": W.hb_shaped,
             "photon_plane_81x51_d4131": W.photon_plane, "hb_two_bonds_d4096": W.hb_two_bonds}[wl]()
        steps = args.qme_steps or m["n_steps"]
        t_build = time.perf_counter()
        gm = qed.Model(m, precision=prec, scheme=args.scheme)
        # basis, operators and U = exp(-i H dt) (the "Taylor approximation" stage of Table 3)
        extra["model_build_s"] = time.perf_counter() - t_build
        D = gm.dim
        rho0 = torch.zeros((D, D), dtype=torch.complex128, device=dev)
        i0 = gm.initial_index()
        rho0[i0, i0] = 1.0
        rho = rho0.clone()
        if wl == "adjoint_lattice_24x24_d1153":
            # loss weights: the photon and the atom population of the corner cavity (0, 0)
            photon, atom, _ = qed.digit_positions(m)
            w = torch.zeros(D, dtype=torch.float64, device=dev)
            for pos in (photon[0], atom[0]):
                d = np.zeros(gm.n_digits, dtype=np.int32)
                d[pos] = 1
                w[gm.index_of(d)] = 1.0

            def one():
                gm.adjoint(rho0, steps, w, checkpoint_every=m["checkpoint_every"])
            unit = "adjoint QME steps/s"
        elif wl == "selection_hb_shaped_d512":
            # the whole trajectory as rounds of state space selection (Sec. 3.2)
            per_round = args.selection_round
            rounds = max(1, steps // per_round)
            steps = rounds * per_round
            final = {}

            def one():
                red, _, keep, sizes = qed.select_states(gm, rho0, per_round, rounds, args.selection_eps)
                final["dim"] = int(red.dim)
                final["sizes_first"] = [int(x) for x in sizes[:3]]
                red.close()
            unit = "QME steps/s"
            extra["selection"] = {"eps": args.selection_eps, "steps_per_round": per_round, "rounds": rounds,
                                  "result": final}
        else:
            r = m["record_every"]
            rec = torch.zeros((gm.n_records(steps, r), D), dtype=torch.float64, device=dev)

            def one():
                rho.copy_(rho0)
                gm.evolve(rho, steps, record_every=r, obs_ids=list(range(D)), records=rec)
            unit = "QME steps/s"
        # the selection run's dimension shrinks as it goes: no per-step flop count
        flops = 0.0 if wl == "selection_hb_shaped_d512" else 16.0 * D ** 3
        per_step_units = steps
        extra["dim"] = D
    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = qed.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        one()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    launches = qed.launch_count() - launches0
    clocks = sampler.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    value = args.steps * per_step_units / (t_ms / 1e3)
    qme_rate = args.steps * steps / (t_ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16x2->f32 (split), f64 master" if prec != "fp64" else "f64", "data": "synthetic",
        "config": dict({"workload": wl, "qme_steps_per_step": steps, "precision": prec, "scheme": args.scheme,
                        "l2": "flushed (512 MB write) between timed iterations"}, **extra),
        "complex_tflops": flops * qme_rate / 1e12, "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload != WORKLOAD:
        run_other(a)
    else:
        run_ours(a)
