"""Benchmark of the MD + MDLG hot path on GB300.

Workload: the production 2D Lennard-Jones gas, N = 4 194 304 at rho = 0.3,
T = 1 (L = 3740, rounded up to a multiple of dx = 4), eps = sigma = m = 1,
rc = 2.5 truncated-shifted, dt = 0.005; MDLG binning at dx = 4 for the coarse
time steps 10, 20, 50, 100 and 200 MD steps; FP64 energy / momentum / virial
reductions every 100 steps.  One benchmark step = 200 MD steps (all lags bin at
least once, sorts included).  Metric: particle-steps per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (launched by torch.distributed.run): one independent system per rank
(different seed), no data-path collective ("scaling": "weak").
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import mdlg_inputs as mi  # noqa: E402

MD_STEPS_PER_STEP = 200
METRIC = "MD+MDLG particle-steps/s on 1 GB300 (% FP32/HBM roofline); batched & adjoint vs plain"
UNIT = "particle-steps/s"
# algorithmic bytes of one particle-step of the fused force + velocity-Verlet
# kernel: positions read and written (12 B each: two 16-bit cell ids + two
# binary32 offsets) and velocities read and written (8 B each); the layout here
# reads a 32-bit cell word and does not write it back (36 B moved)
STEP_BYTES_PER_PARTICLE = 40
IDEALGAS_BYTES_PER_PARTICLE = 16  # x, y, vx, vy binary32
COLLISION_BYTES_PER_SITE_Q = 12   # read n_i at x and at x + v_i, write Xi_i: 3 x 4 B per velocity
COLLISION_BYTES_PER_SITE = 12     # dmass + dmom int32
FP32_LANES_PER_SM = 128
SMSP_PER_SM = 4


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def _traffic_record(kernel: str, key: str = "dram_bytes_per_particle"):
    """A per-particle counter of a kernel (DRAM bytes, warp instructions) from
    profiles/traffic.txt, if the kernel source has not changed since that
    capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        import hashlib
        src = open(os.path.join(ROOT, "paper_1705_04368_gb300", "csrc", "mdlg_md.cu"), "rb").read()
        sha = hashlib.sha256(src).hexdigest()[:16]
        for ln in open(path):
            kv = dict(t.split("=", 1) for t in ln.split() if "=" in t)
            if kv.get("kernel") == kernel and kv.get("src_sha") == sha and key in kv:
                return float(kv[key])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[3 + k].lower() in ("active", "1")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def rank_seed(rank: int) -> int:
    """Seed of the independent system a rank advances (weak scaling: one system each)."""
    return 1 + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest of every rank's value (a job takes as long as its slowest rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world * units_per_rank / seconds


def _workload():
    c = mi.PRODUCTION_LJ
    return c


def _config(c, world):
    rho_eff = c.n / (c.box * c.box)
    return {"workload": c.name, "n": c.n, "box": c.box, "rho_eff": round(rho_eff, 5),
            "temperature": c.temperature, "rc": c.rc, "dt": c.dt, "dx": c.dx,
            "lag_md_steps": list(c.lags), "md_steps_per_step": MD_STEPS_PER_STEP,
            "stats_every": 100, "systems": world,
            "l2": "inputs larger than L2 (state 352 MB per system, 151 MB moved per MD step)"}


def _params(c, m):
    return m.Params(n=c.n, box=c.box, dx=c.dx, dt=c.dt, lag_steps=c.lags, rcut=c.rc,
                    stats_every=100)


def _cpu_info():
    """Host core count and CPU model (the oracle baselines run on these cores)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model}


def run_oracle_timing(threads: int):
    """The FP64 oracle, as it stands, on the three workloads of the measurement
    plan; one JSON line.  threads = 1: the serial build; 0: the threaded build on
    every host core.  c1: N = 1024 LJ gas, 2000 steps with a binning every 50;
    c3: 3 velocity-Verlet steps of the production gas plus one binning (per
    particle-step); c2: one snapshot of the 2^22-particle ideal gas, 9 pairs."""
    import oracle
    used = 1 if threads == 1 else oracle.use_threads(threads)
    out = {"threads": used, **_cpu_info()}
    c = mi.SMALL_LJ
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=1)
    t0 = time.perf_counter()
    ref = oracle.VV(x0, v0, (c.box, c.box), c.dt, cells=True)
    cnt = np.zeros(50, np.uint64)
    cells = (int(c.box / c.dx),) * 2
    prev = ref.x.copy()
    for _ in range(c.steps // c.lags[0]):
        ref.run(c.lags[0])
        oracle.mdlg_bin(prev, ref.x, c.dx, cells, c.vmax, counts=cnt)
        prev = ref.x.copy()
    s1 = time.perf_counter() - t0
    out["c1"] = {"workload": c.name, "md_steps": c.steps, "seconds": s1,
                 "particle_steps_per_s": c.n * c.steps / s1}
    c = mi.PRODUCTION_LJ
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=1)
    k = 3
    t0 = time.perf_counter()
    ref = oracle.VV(x0, v0, (c.box, c.box), c.dt, cells=True)
    ref.run(k)
    oracle.mdlg_bin(x0, ref.x, c.dx, (int(c.box / c.dx),) * 2, 3, counts=np.zeros(50, np.uint64))
    s3 = time.perf_counter() - t0
    out["c3"] = {"workload": c.name, "md_steps": k, "seconds": s3,
                 "particle_steps_per_s": c.n * k / s3}
    pos, vel = mi.idealgas_state(mi.IDEALGAS_N, mi.IDEALGAS_BOX, 1.0, seed=7)
    combos = list(mi.IDEALGAS_COMBOS)
    t0 = time.perf_counter()
    oracle.stream_bin_f32(pos, vel, [x[0] for x in combos], [x[1] for x in combos], 3)
    s2 = time.perf_counter() - t0
    out["c2"] = {"workload": "idealgas_n4194304_L2048_9combos", "seconds": s2,
                 "particles_per_s": mi.IDEALGAS_N / s2}
    print(json.dumps(out), flush=True)


def _oracle_timings():
    """run_oracle_timing in child processes (one loads the serial build, one the
    threaded build): single thread, then every host core."""
    res = {}
    for name, th in (("one_thread", 1), ("all_cores", 0)):
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-timing", str(th)],
                           capture_output=True, text=True, timeout=900)
        if r.returncode != 0:
            res[name] = {"error": r.stderr.strip().splitlines()[-1:] or [f"rc {r.returncode}"]}
            continue
        res[name] = json.loads(r.stdout.strip().splitlines()[-1])
    return res


def run_reference(args, rank, world):
    if rank != 0:
        return
    c = _workload()
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=1)
    import oracle
    cores = oracle.use_threads(0)
    ref = oracle.VV(x0, v0, (c.box, c.box), c.dt, cells=True)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ref.run(1)
        dt_s = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt_s)
    total = sum(times)
    value = c.n * len(times) / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(c, 1),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{len(times)} bench steps of one FP64 velocity-Verlet "
                                       f"step each (not 200) of the full {c.n}-particle "
                                       f"system, linked-cell oracle, {cores} host threads",
                             **_cpu_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1705_04368_gb300 as m

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = _workload()
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=rank_seed(rank))
    stream = torch.cuda.Stream(device=dev)
    # neighbour-cell geometry picked by the autotuner (cached per workload; untimed)
    from paper_1705_04368_gb300 import tune
    params, tune_report = tune.tune(_params(c, m), x0, v0, c.temperature)
    sim = m.Simulation(params, x0, v0, stream=stream, device=local_rank)
    for _ in range(args.warmup):
        sim.step(MD_STEPS_PER_STEP)
    torch.cuda.synchronize()

    dist = None
    if world > 1:
        import torch.distributed as dist
    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sim.profile(True)
    e0.record(stream)
    for _ in range(args.steps):
        sim.step(MD_STEPS_PER_STEP)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = sim.profile(False)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    st, counts, fi = sim.stats()
    sim.close()
    md_steps = args.steps * MD_STEPS_PER_STEP
    value = job_rate(world, c.n * md_steps, ms / 1e3)

    # roofline denominators: HBM from MEASURED_PEAKS.json, FP32 from the project's
    # FMA probe (the copy probe is reported beside the HBM figure as a cross-check)
    hbm_gbs, sm_max_mhz, peak_kind = _peaks()
    probes = _probe_peaks(m, torch, dev, stream)
    sms = probes["sms"]
    fp32_nominal = sms * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    fp32_peak = probes["fp32_tflops"]
    probes["fp32_tflops_nominal"] = fp32_nominal
    probes["hbm_gbs_measured_peaks"] = hbm_gbs
    # dominant kernel: fused force + velocity-Verlet step
    step_ms, step_launches = prof["step"]
    avg_step_s = step_ms / 1e3 / max(step_launches, 1)
    rho_eff = c.n / (c.box * c.box)
    roofline = _step_roofline(c.n, rho_eff, c.rc, avg_step_s, hbm_gbs, fp32_peak, peak_kind)
    tpp = _traffic_record("k_step_loop")
    ipp = _traffic_record("k_step_loop", "warp_inst_per_particle")
    roofline["traffic"] = (tpp * c.n) if tpp is not None else None
    # instruction issue: one warp instruction per clock per SM sub-partition
    issue_peak = sms * SMSP_PER_SM * sm_max_mhz * 1e6
    roofline["issue"] = None if ipp is None else {
        "achieved_warp_inst_per_s": ipp * c.n / avg_step_s,
        "peak_warp_inst_per_s": issue_peak,
        "frac": ipp * c.n / avg_step_s / issue_peak,
        "warp_inst_per_particle": ipp,
        "what": "ncu warp-instruction count of one launch (profiles/traffic.txt) over the launch "
                "time measured here; peak = one issue per clock per SM sub-partition at the "
                "maximum SM clock"}
    kernels = {k: {"ms": v[0], "launches": v[1], "share": v[0] / ms if ms else None}
               for k, v in prof.items() if v[1]}
    launches = prof["step"][1] + prof["sort"][1] + prof["bin"][1] + prof["sync"][1]

    # the dense production case (rho = 0.6, T = 0.8) with its own roofline
    dense = _production_leg(m, torch, stream, local_rank, mi.PRODUCTION_LJ_DENSE, rank_seed(rank),
                            hbm_gbs, fp32_peak, peak_kind) if rank == 0 else None
    # the small case (N = 1024), absolute time only
    small = _small_leg(m, torch, stream, local_rank) if rank == 0 else None

    # ideal-gas single pass (binning throughput), rotating buffers > 2x L2
    ig = _idealgas(m, torch, dev, stream, hbm_gbs)

    # batched replicas (256 systems) against the same systems one context at a time
    batched = _batched(m, torch, stream, local_rank) if rank == 0 else None

    # adjoint (N = 16 384, rho = 0.3, K = 200, checkpoints every 20) versus the plain forward
    adjoint = _adjoint(m, torch, stream, local_rank) if rank == 0 else None

    # paper analyses: collision-operator kernel alone, and the production run
    # with the moving lattice, Xi field and mean-square displacement switched on
    analyses = _analyses(m, torch, dev, stream, local_rank, params, c, x0, v0, hbm_gbs, value / world) \
        if rank == 0 else None
    if analyses:
        analyses["production_with_analyses"]["plain_bin_ms_per_200_steps"] = prof["bin"][0] / args.steps

    # end to end through the C ABI: pinned host state in, f_i out, every step
    e2e = _e2e(m, torch, params, c, x0, v0, stream, local_rank, args, world, dist, dev)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": _config(c, world), "roofline": roofline,
            "gpu_launches": launches, "kernels": kernels, "clocks": clk, "e2e": e2e,
            "idealgas": ig, "batched": batched, "adjoint": adjoint, "analyses": analyses,
            "dense": dense, "small": small, "peaks": probes,
            "status": st["status"],
            "tuned": {"grid": params.grid, "skin": params.skin,
                      "cell_width": params.grid * math.ceil((params.rcut + params.skin) / params.grid - 1e-12),
                      "cached": tune_report["cached"]}}
    if rank == 0:
        if world == 1:
            ot = _oracle_timings()
            line["oracle_timings"] = ot
            allc = ot.get("all_cores", {})
            one = ot.get("one_thread", {})
            if "c3" in allc:
                line["cpu_baseline"] = {
                    "value": allc["c3"]["particle_steps_per_s"], "unit": UNIT,
                    "cores": allc["threads"], "kind": "oracle",
                    "sample": f"3 FP64 velocity-Verlet steps of the full {c.n}-particle system "
                              f"plus one MDLG binning, {allc['c3']['seconds']:.1f} s on "
                              f"{allc['threads']} host threads (threaded build of the oracle)",
                    "nproc": allc.get("nproc"), "cpu_model": allc.get("model"),
                    "one_thread": one.get("c3")}
        print(json.dumps(line), flush=True)


def _probe_peaks(m, torch, dev, stream):
    """FP32 multiply-add rate and HBM copy bandwidth measured with the library's
    probe kernels (CUDA events on the library's stream): the FMA loop on every SM
    (8 blocks of 256 threads per SM, 8 independent chains per thread), the copy
    over two 512 MiB buffers (4x L2 each), best of several launches."""
    import ctypes
    lib = m.lib()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads, iters = sms * 8, 256, 1 << 18
    out = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    fl = ctypes.c_double()
    h = stream.cuda_stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def best_of(fn, reps):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return best

    def fma():
        assert lib.mdlg_probe_fma(blocks, threads, iters, out.data_ptr(), ctypes.byref(fl), h) == 0

    t_fma = best_of(fma, 3)
    nbytes = 512 << 20
    src = torch.empty(nbytes // 4, dtype=torch.int32, device=dev)
    dst = torch.empty_like(src)

    def copy():
        assert lib.mdlg_probe_copy(src.data_ptr(), dst.data_ptr(), nbytes, h) == 0

    t_copy = best_of(copy, 10)
    del src, dst, out
    return {"sms": sms, "fp32_tflops": fl.value / t_fma / 1e12,
            "hbm_copy_gbs": 2 * nbytes / t_copy / 1e9,
            "what": "mdlg_probe_fma: 8 blocks x 256 threads per SM, 8 independent binary32 FMA "
                    "chains per thread; mdlg_probe_copy: 512 MiB copied with 16-byte words "
                    "(read + write bytes); best of 3 / 10 launches"}


def _step_roofline(n, rho_eff, rc, avg_step_s, hbm_gbs, fp32_peak, peak_kind):
    """The fused force + velocity-Verlet kernel against HBM (40 B per particle-step)
    and against the FP32 peak (18 n_in + 8 flops per particle-step, n_in = rho pi rc^2),
    with the FP32 fraction the HBM roofline allows at this density."""
    step_bytes = STEP_BYTES_PER_PARTICLE * n
    achieved_gbs = step_bytes / avg_step_s / 1e9
    n_in = rho_eff * math.pi * rc ** 2
    fpp = 18.0 * n_in + 8.0
    achieved_tf = n * fpp / avg_step_s / 1e12
    intensity = fpp / STEP_BYTES_PER_PARTICLE
    cap = min(1.0, intensity * hbm_gbs / 1e3 / fp32_peak)
    return {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_gbs, "unit": "GB/s",
            "frac": achieved_gbs / hbm_gbs, "peak_kind": peak_kind,
            "kernel": "k_step_loop (force + velocity-Verlet; k_step on statistics steps)",
            "algorithmic_bytes_per_launch": step_bytes, "avg_launch_us": avg_step_s * 1e6,
            "fp32": {"achieved_tflops": achieved_tf, "peak_tflops": fp32_peak,
                     "frac": achieved_tf / fp32_peak, "flops_per_particle": fpp,
                     "intensity_flop_per_byte": intensity,
                     "cap_frac_at_hbm_peak": cap,
                     "frac_of_cap": achieved_tf / fp32_peak / cap}}


def _production_leg(m, torch, stream, local_rank, c, seed, hbm_gbs, fp32_peak, peak_kind,
                    steps=2):
    """Another production configuration (tuned geometry, 200 MD steps per bench
    step, binning and statistics as in the headline leg), timed with CUDA events."""
    from paper_1705_04368_gb300 import tune
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=seed)
    params, rep = tune.tune(_params(c, m), x0, v0, c.temperature)
    with m.Simulation(params, x0, v0, stream=stream, device=local_rank) as s:
        s.step(MD_STEPS_PER_STEP)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.profile(True)
        e0.record(stream)
        for _ in range(steps):
            s.step(MD_STEPS_PER_STEP)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = s.profile(False)
        st, _, _ = s.stats()
    ms = e0.elapsed_time(e1)
    step_ms, nst = prof["step"]
    rho_eff = c.n / (c.box * c.box)
    return {"workload": c.name, "n": c.n, "box": c.box, "rho_eff": round(rho_eff, 5),
            "temperature": c.temperature, "status": st["status"],
            "particle_steps_per_s": c.n * steps * MD_STEPS_PER_STEP / (ms / 1e3),
            "ms_per_step": ms / steps,
            "tuned": {"grid": params.grid, "skin": params.skin, "cached": rep["cached"]},
            "kernels": {k: {"ms": v[0], "launches": v[1], "share": v[0] / ms}
                        for k, v in prof.items() if v[1]},
            "roofline": _step_roofline(c.n, rho_eff, c.rc, step_ms / 1e3 / max(nst, 1), hbm_gbs,
                                       fp32_peak, peak_kind)}


def _small_leg(m, torch, stream, local_rank):
    """The small LJ gas (N = 1024, L = 64, dx = 4, lag 50): 2000 MD steps and the
    statistics read-back, wall time (the size is launch-bound; CUDA graphs on)."""
    c = mi.SMALL_LJ
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=1)
    p = m.Params(n=c.n, box=c.box, dx=c.dx, dt=c.dt, lag_steps=c.lags, use_graphs=True)
    with m.Simulation(p, x0, v0, stream=stream, device=local_rank) as s:
        s.step(c.steps)           # captures the schedule's graph
        s.stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(c.steps)
        st, _, _ = s.stats()
        sec = time.perf_counter() - t0
    return {"workload": c.name, "md_steps": c.steps, "seconds": sec,
            "particle_steps_per_s": c.n * c.steps / sec, "status": st["status"]}


def _idealgas(m, torch, dev, stream, hbm_gbs):
    n = mi.IDEALGAS_N
    combos = list(mi.IDEALGAS_COMBOS)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    bufs = []
    with torch.cuda.stream(stream):
        for _ in range(4):
            pos = (1.0 - torch.rand((n, 2), generator=g, device=dev)) * mi.IDEALGAS_BOX
            vel = torch.randn((n, 2), generator=g, device=dev)
            bufs.append((pos.float().contiguous(), vel.float().contiguous()))
        counts = torch.zeros((len(combos), 50), dtype=torch.int64, device=dev)
    for k in range(4):
        m.idealgas_bin(*bufs[k % 4], combos, 3, counts, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 40
    e0.record(stream)
    for k in range(reps):
        m.idealgas_bin(*bufs[k % 4], combos, 3, counts, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3 / reps
    gbs = n * IDEALGAS_BYTES_PER_PARTICLE / s / 1e9
    return {"workload": "idealgas_n4194304_L2048_9combos", "particles_per_s": n / s,
            "us_per_pass": s * 1e6, "achieved_gbs": gbs, "frac_hbm": gbs / hbm_gbs,
            "bin_decisions_per_s": n * len(combos) / s}


def _batched(m, torch, stream, local_rank, md_steps=700):
    """256 replicas (N log-uniform in [1k, 64k], rho uniform in [0.1, 0.6], T = 1,
    dx = 4, lag 50): particle-steps/s advanced as one batch versus one context per
    system.  Each arm runs the schedule that suits it: the batch launches directly
    with device-paced re-sorts (its steps take ~0.2 ms, so launches are cheap); the
    single contexts, whose steps are launch-bound, replay CUDA graphs of a 700-step
    schedule with a re-sort every 7 steps (captured during an untimed first pass)."""
    from paper_1705_04368_gb300 import tune
    ns, boxes, seeds = mi.batch_recipe()
    x0, v0 = mi.batch_states(ns, boxes, seeds)
    params = m.Params(n=0, box=64.0, dx=4.0, lag_steps=(50,), sort_every=0)
    # neighbour-cell geometry tuned for the whole batch (untimed)
    params, trep = tune.tune_batch(params, ns, boxes, x0, v0, 1.0)
    total = int(ns.sum())
    with m.BatchSimulation(params, ns, boxes, x0, v0, stream=stream, device=local_rank) as bt:
        bt.step(md_steps)          # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.step(md_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t_batch = e0.elapsed_time(e1) / 1e3
        st, _, _ = bt.stats()
    sims, off = [], 0
    for n, b in zip(ns, boxes):
        p = m.Params(n=int(n), box=float(b[0]), dx=4.0, lag_steps=(50,), sort_every=7,
                     use_graphs=True, grid=params.grid, skin=params.skin)
        sims.append(m.Simulation(p, x0[off:off + n], v0[off:off + n], stream=stream,
                                 device=local_rank))
        off += int(n)
    for sm in sims:
        sm.step(md_steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sm in sims:
        sm.step(md_steps)
    torch.cuda.synchronize()
    t_alone = time.perf_counter() - t0
    for sm in sims:
        sm.close()
    return {"workload": "lj2d_batch256_n1k-64k_rho0.1-0.6_T1", "systems": len(ns),
            "particles": total, "md_steps": md_steps,
            "schedules": "batch: direct launches, device-paced re-sorts; one context each: "
                         "CUDA graphs, re-sort every 7 steps",
            "batched_particle_steps_per_s": total * md_steps / t_batch,
            "one_context_each_particle_steps_per_s": total * md_steps / t_alone,
            "speedup": t_alone / t_batch, "status": st["status"],
            "tuned": {"grid": params.grid, "skin": params.skin, "cached": trep["cached"],
                      "candidates": trep.get("candidates")}}


def _adjoint(m, torch, stream, local_rank, reps=3):
    """Seconds for the gradient of the soft-binned second moment over 200 steps
    (shifted-force LJ, N = 16 384, rho = 0.3, T = 1, checkpoints every 20) against
    the plain 200-step forward of the same system."""
    n, K, ck = 16384, 200, 20
    L = mi.box_for(n, 0.3, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=16387)
    vel = np.array([(vx, vy) for vy in range(-3, 4) for vx in range(-3, 4)], np.float64)
    w = (vel ** 2).sum(axis=1)
    p = m.Params(n=n, box=L, dx=4.0, sort_every=ck, potential=m.POT_LJ_SF)

    def run(kind):
        with m.Simulation(p, x0, v0, stream=stream, device=local_rank) as s:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if kind == "forward":
                s.step(K)
                s.stats()
            else:
                s.adjoint(K, ck, 2.0, dloss=w)
            torch.cuda.synchronize()
            return time.perf_counter() - t0

    run("forward"), run("adjoint")            # warm up
    tf = min(run("forward") for _ in range(reps))
    ta = min(run("adjoint") for _ in range(reps))
    return {"workload": "lj2d_sf_n16384_rho0.3_T1_K200_ckpt20", "forward_s": tf,
            "adjoint_s": ta, "adjoint_over_forward": ta / tf,
            "what": "mdlg_adjoint with gradients (forward with checkpoints, segment "
                    "recompute, reverse sweep, soft loss) vs mdlg_step(200) + mdlg_stats"}


def _analyses(m, torch, dev, stream, local_rank, params, c, x0, v0, hbm_gbs, plain_value, reps=20):
    """(1) mdlg_collision on the production lattice (935 x 935 sites, V = 3) with
    random fields, algorithmic bytes 12 Q + 12 per site; (2) the production run
    (200 MD steps per step) with lattice drift U = (0.3, 0.1), the Xi field of
    lag 0, and the mean-square displacement and velocity correlation of every
    lag, against the plain run."""
    import dataclasses
    C = (int(round(c.box / c.dx)),) * 2
    q = 49
    sites = C[0] * C[1]
    g = torch.Generator(device=dev)
    g.manual_seed(11)
    with torch.cuda.stream(stream):
        fields = [torch.randint(0, 20, (sites, q + 1), generator=g, device=dev, dtype=torch.int32)
                  for _ in range(3)]
        xi = torch.empty((sites, q), dtype=torch.int32, device=dev)
        dm = torch.empty(sites, dtype=torch.int32, device=dev)
        dj = torch.empty((sites, 2), dtype=torch.int32, device=dev)
    for k in range(3):
        m.collision(C, 3, fields[k % 3], fields[(k + 1) % 3], xi, dm, dj, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(reps):
        m.collision(C, 3, fields[k % 3], fields[(k + 1) % 3], xi, dm, dj, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_coll = e0.elapsed_time(e1) / 1e3 / reps
    coll_bytes = sites * (COLLISION_BYTES_PER_SITE_Q * q + COLLISION_BYTES_PER_SITE)
    del fields, xi, dm, dj

    p = dataclasses.replace(params, lattice_u=(0.3, 0.1), msd=True, vacf=True,
                            site_mode=m.SITES_FIELD | m.SITES_XI)
    with m.Simulation(p, x0, v0, stream=stream, device=local_rank) as s:
        s.step(MD_STEPS_PER_STEP)
        torch.cuda.synchronize()
        s.profile(True)
        e0.record(stream)
        for _ in range(3):
            s.step(MD_STEPS_PER_STEP)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = s.profile(False)
        st, _, _ = s.stats()
    t_run = e0.elapsed_time(e1) / 1e3
    on_value = c.n * 3 * MD_STEPS_PER_STEP / t_run
    return {"collision": {"workload": f"lattice_{C[0]}x{C[1]}_V3", "us_per_launch": t_coll * 1e6,
                          "algorithmic_bytes": coll_bytes,
                          "achieved_gbs": coll_bytes / t_coll / 1e9,
                          "frac_hbm": coll_bytes / t_coll / 1e9 / hbm_gbs},
            "production_with_analyses": {
                "lattice_u": st["lattice_u"], "msd_lag0": st["msd"][0], "status": st["status"],
                "particle_steps_per_s": on_value, "plain_particle_steps_per_s": plain_value,
                "overhead": plain_value / on_value - 1.0,
                "bin_ms_per_200_steps": prof["bin"][0] / 3, "bin_launches": prof["bin"][1],
                "vacf_lag0": st["vacf"][0],
                "what": "moving lattice + SITES_FIELD|SITES_XI + msd + vacf, graphs off (both arms)"}}


def _e2e(m, torch, params, c, x0, v0, stream, local_rank, args, world, dist, dev):
    x_pin = torch.empty((c.n, 2), dtype=torch.float64, pin_memory=True)
    v_pin = torch.empty((c.n, 2), dtype=torch.float64, pin_memory=True)
    x_pin.numpy()[:] = x0
    v_pin.numpy()[:] = v0
    reps = max(2, min(args.steps, 5))

    def one():
        with m.Simulation(params, x_pin.numpy(), v_pin.numpy(), stream=stream,
                          device=local_rank) as s:
            s.step(MD_STEPS_PER_STEP)
            s.stats()

    one()   # warm the allocator
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(reps):
        one()
    torch.cuda.synchronize()
    secs = max_over_ranks(time.perf_counter() - t0, dist, dev)
    q1 = params.q1
    nl = len(params.lag_steps)
    return {"value": job_rate(world, c.n * MD_STEPS_PER_STEP * reps, secs), "unit": UNIT,
            "h2d_bytes_per_step": 2 * c.n * 2 * 8,
            "d2h_bytes_per_step": 2 * nl * q1 * 8 + 120,
            "steps": reps,
            "what": "mdlg_create from pinned host x0, v0 + 200 MD steps + mdlg_stats (counts, "
                    "f_i to host) + mdlg_destroy, per step"}


def run_ncu_target(md_steps, dense=False):
    """profiling target (ncu --profile-from-start off): the bench's production
    system (dense: the rho = 0.6, T = 0.8 case) with the tuned geometry, one
    untimed bench step, then md_steps MD steps between cudaProfilerStart and
    cudaProfilerStop -- the launch mix of the timed region."""
    import torch
    import paper_1705_04368_gb300 as m
    from paper_1705_04368_gb300 import tune
    c = mi.PRODUCTION_LJ_DENSE if dense else _workload()
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=1)
    params, _ = tune.tune(_params(c, m), x0, v0, c.temperature)
    sim = m.Simulation(params, x0, v0)
    sim.step(MD_STEPS_PER_STEP)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    sim.step(md_steps)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    sim.close()


def run_state_point(total: int, discard: int):
    """The paper's own state point on this engine (Sec. IV, Figs. VD and wi_u):
    N = 100 000, L = 1000 sigma, T = 50, dt = 1e-4; `total` MD steps of which the
    first `discard` are dropped (the paper: 3e6 and 1e6).  Lattice dx = 100 sigma,
    coarse step dt_LG = 34.16 tau (341 600 MD steps), imposed lattice velocity u =
    0 ... 0.5 (lattice units) by moving the lattice; the MSD of six shorter lags
    gives the decay time tau of Eq. vca, and their velocity correlation (u = 0)
    gives it a second time, from T exp(-t/tau) at the lags up to 0.7 tau
    (Fig. VD(a)).  Prints one JSON line: per u the
    measured f_i against Eq. feqfull (at the measured a^2) and against the D2Q9
    equilibrium of Eq. f0lb (theta = 1/3)."""
    import torch
    import paper_1705_04368_gb300 as m
    from paper_1705_04368_gb300 import analysis as an
    c = mi.PAPER_STATE_POINT
    dx, lag = 100.0, 341_600
    lags = (100, 1000, 3000, 7000, 20000, 50000, lag)
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=5)
    out = {"workload": "lj2d_n100000_L1000_T50_dt1e-4", "md_steps": total, "discarded": discard,
           "dx": dx, "dt_lattice_tau": lag * c.dt, "runs": []}
    t0 = time.perf_counter()
    for u in (0.0, 0.1, 0.2, 0.3, 0.4, 0.5):
        U = u * dx / (lag * c.dt)
        p = m.Params(n=c.n, box=c.box, dx=dx, dt=c.dt, lag_steps=lags, vmax=c.vmax, msd=True,
                     vacf=(u == 0.0), stats_every=10000, lattice_u=(U, 0.0))
        with m.Simulation(p, x0, v0) as s:
            s.step(discard)
            s.reset_counts()
            s.step(total - discard)
            st, _, fi = s.stats()
        torch.cuda.synchronize()
        T = st["temperature"]
        msd = [0.5 * (a + b) for a, b in st["msd"]]
        if u == 0.0:
            ts = [l * c.dt for l in lags[:-1]]
            grid = np.linspace(0.1, 1.5, 1401)
            err = [sum((math.log(an.msd_exponential(T, tau, t)) - math.log(mm)) ** 2
                       for t, mm in zip(ts, msd)) for tau in grid]
            out["tau_fit"] = float(grid[int(np.argmin(err))])
            out["temperature"] = T
            # Fig. VD(a): the velocity correlation per lag, and the decay time of
            # T exp(-t/tau) fitted to the lags up to 0.7 tau
            vc = [0.5 * (a + b) for a, b in st["vacf"][:-1]]
            out["vacf_over_T"] = {f"{t:g}": cv / T for t, cv in zip(ts, vc)}
            early = [(t, cv) for t, cv in zip(ts, vc) if t <= 0.7 + 1e-12 and cv > 0]
            err = [sum((math.log(cv / T) + t / tau) ** 2 for t, cv in early) for tau in grid]
            out["tau_fit_vacf"] = float(grid[int(np.argmin(err))])
        ueff = st["lattice_u"][0] * lag * c.dt / dx
        a = math.sqrt(msd[-1]) / dx
        f = fi[-1]
        th = an.feq(c.vmax, a, (ueff, 0.0))
        lb = an.lb_equilibrium((ueff, 0.0), vmax=c.vmax)
        shell = np.abs(an.velocity_table(c.vmax)).max(axis=1) <= 1
        w = 2 * c.vmax + 1
        pick = {"rest": (0, 0), "east": (1, 0), "west": (-1, 0), "north": (0, 1),
                "north_east": (1, 1), "north_west": (-1, 1)}
        out["runs"].append({
            "u": ueff, "a2": a * a, "intervals": st["intervals"][-1], "status": st["status"],
            "max_abs_vs_closed_form": float(np.abs(f[:-1] - th[:-1]).max()),
            "max_abs_vs_lb_one_shell": float(np.abs(f[:-1][shell] - lb[:-1][shell]).max()),
            "mean_velocity": float(an.moments(f, c.vmax)["mean"][0]),
            "f": {k: [float(f[(vy + c.vmax) * w + vx + c.vmax]),
                      float(th[(vy + c.vmax) * w + vx + c.vmax]),
                      float(lb[(vy + c.vmax) * w + vx + c.vmax])] for k, (vx, vy) in pick.items()}})
    out["seconds"] = time.perf_counter() - t0
    print(json.dumps(out), flush=True)


def run_ncu_collision(launches):
    """profiling target: the collision operator on the production lattice
    (935 x 935 sites, V = 3, random fields), `launches` launches."""
    import torch
    import paper_1705_04368_gb300 as m
    dev = torch.device("cuda", 0)
    C = (935, 935)
    g = torch.Generator(device=dev)
    g.manual_seed(11)
    f = [torch.randint(0, 20, (C[0] * C[1], 50), generator=g, device=dev, dtype=torch.int32)
         for _ in range(2)]
    xi = torch.empty((C[0] * C[1], 49), dtype=torch.int32, device=dev)
    dm = torch.empty(C[0] * C[1], dtype=torch.int32, device=dev)
    dj = torch.empty((C[0] * C[1], 2), dtype=torch.int32, device=dev)
    for k in range(launches):
        m.collision(C, 3, f[k % 2], f[(k + 1) % 2], xi, dm, dj)
    torch.cuda.synchronize()


def run_ncu_idealgas(launches):
    """profiling target: `launches` ideal-gas passes over the 2^22-particle gas
    (9 (dx, dt) pairs), the bench's idealgas leg."""
    import torch
    import paper_1705_04368_gb300 as m
    dev = torch.device("cuda", 0)
    pos, vel = mi.idealgas_state(mi.IDEALGAS_N, mi.IDEALGAS_BOX, 1.0, seed=7)
    pos, vel = torch.from_numpy(pos).to(dev), torch.from_numpy(vel).to(dev)
    counts = torch.zeros((len(mi.IDEALGAS_COMBOS), 50), dtype=torch.int64, device=dev)
    for _ in range(launches):
        m.idealgas_bin(pos, vel, list(mi.IDEALGAS_COMBOS), 3, counts)
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--ncu-target", type=int, default=0, metavar="MD_STEPS",
                    help="profiling target: the production system after one untimed bench "
                         "step, MD_STEPS MD steps inside cudaProfilerStart/Stop, exit")
    ap.add_argument("--ncu-dense", action="store_true",
                    help="with --ncu-target: the rho = 0.6, T = 0.8 production case")
    ap.add_argument("--ncu-collision", type=int, default=0, metavar="LAUNCHES",
                    help="profiling target: LAUNCHES collision-operator launches on the "
                         "production lattice, exit")
    ap.add_argument("--state-point", type=int, nargs=2, default=None, metavar=("TOTAL", "DISCARD"),
                    help="the paper's state point (N = 100 000, T = 50): TOTAL MD steps, the first "
                         "DISCARD dropped (the paper: 3000000 1000000); u-sweep of the moving "
                         "lattice at dx = 100, dt_LG = 34.16; one JSON line")
    ap.add_argument("--ncu-idealgas", type=int, default=0, metavar="LAUNCHES",
                    help="profiling target: LAUNCHES ideal-gas passes, exit")
    ap.add_argument("--oracle-timing", type=int, default=None, metavar="THREADS",
                    help="time the FP64 oracle on the measurement plan's CPU samples (1: serial "
                         "build, 0: threaded build on every core); one JSON line, exit")
    args = ap.parse_args()
    if args.oracle_timing is not None:
        run_oracle_timing(args.oracle_timing)
        return
    if args.ncu_idealgas:
        run_ncu_idealgas(args.ncu_idealgas)
        return
    if args.state_point:
        run_state_point(*args.state_point)
        return
    if args.ncu_collision:
        run_ncu_collision(args.ncu_collision)
        return
    if args.ncu_target:
        run_ncu_target(args.ncu_target, dense=args.ncu_dense)
        return
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
