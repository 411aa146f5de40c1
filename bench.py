"""Benchmark of the residual + SSP-RK3 stage on one GB300 (or N replicas).

One step = one SSP-RK3 time step = three (edge flux, divergence + stage)
passes over the 250,000-vertex periodic isentropic-vortex mesh (jittered
500x500 torus lattice split on random diagonals, two-level stencils,
degree-2 least squares, NU-WENO5).  The headline is the FP64 path; beside it
are precision 48 (the same FP64 computation with the edge-flux increments in
double-word FP32 arithmetic) and the FP32 residual path (FP64 state
accumulation), each with its error against FP64.  The same line carries the
adjoint figures of the 250k-vertex adjoint workload (`adjoint`: VJP and
checkpointed-adjoint times against the forward, finite-difference checks)
and the 64-mesh batch (`batch`: one persistent launch per stage, FP32, 48
and 64), each timed in its own region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica on its own GPU (the path has no exchange step); the
time is the max over ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "residual Mvertex/s FP64 vs FP32 at stated error, % HBM roofline; adjoint/fwd time"
N_LATTICE = 500  # 250,000 vertices
CFL = 0.5
# FP64 operations per edge of the edge-flux kernel and per vertex of the
# divergence + stage kernel (counted from the kernel source; FMA = 2).
FLOP_EDGE64 = 631
FLOP_DIV64_PER_VENTRY = 16
FLOP_DIV64_PER_EENTRY = 8
FLOP_DIV64_FIXED = 70
FP64_PEAK_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (non-tensor), NVIDIA datasheet figure
# DRAM bytes per edge of edge_flux_f64 from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum = 121.7 + 7.3 MB on the 480k-edge case of the same
# workload, scaled per edge); None once the kernel changes after the capture.
TRAFFIC_EDGE64_B_PER_EDGE = (121.745408 + 7.27552) * 1e6 / 480000
# From the same capture: FP64 pipe busy (sm__pipe_fp64_cycles_active, % of
# active cycles) and executed FP64 thread instructions (DADD + DFMA + DMUL)
# per edge of edge_flux_f64.
NCU_EDGE64_FP64_PIPE_BUSY = 0.8983
NCU_EDGE64_FP64_INSTR_PER_EDGE = 448.9  # 54.3 DADD + 240.0 DFMA + 154.6 DMUL
# edge_flux_dw (precision 48) from one ncu capture on the 480k-edge case:
# issue slots busy, FMA (FP32) pipe busy, FP64 pipe busy (% of active
# cycles), thread instructions per edge, DRAM bytes per edge.
NCU_EDGE48_ISSUE_ACTIVE = 0.718
NCU_EDGE48_FMA_PIPE = 0.585
NCU_EDGE48_FP64_PIPE = 0.141
NCU_EDGE48_THREAD_INSTR_PER_EDGE = 97722617 * 32 / 480000
TRAFFIC_EDGE48_B_PER_EDGE = (121.78432 + 6.677504) * 1e6 / 480000
# edge_flux_f32 from one ncu capture each on the 480k-edge case: issue slots
# busy, FMA pipe busy, DRAM throughput (% of peak), DRAM bytes per edge; the
# default form (FP64-built block streamed in FP32) and the compact form
# (values formed in the kernel from the stencil gaps, mesh option f32_coef = 1).
NCU_EDGE32_ISSUE_ACTIVE = 0.441
NCU_EDGE32_FMA_PIPE = 0.344
NCU_EDGE32_DRAM = 0.418
TRAFFIC_EDGE32_B_PER_EDGE = (64.013056 + 0.72192) * 1e6 / 480000
NCU_EDGE32G_ISSUE_ACTIVE = 0.644
NCU_EDGE32G_FMA_PIPE = 0.516
NCU_EDGE32G_DRAM = 0.194
TRAFFIC_EDGE32G_B_PER_EDGE = (25.61408 + 0.000512) * 1e6 / 480000


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class _NvmlSampler:
    """SM clock and clocks-event reasons polled through NVML (read-only queries)
    every ~2 ms on a thread, so that a timed region of tens of milliseconds
    still gets many samples.  The device is found by its UUID."""

    # nvmlClocksEventReasons bits (public NVML API)
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, cuda_index):
        import ctypes

        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        import torch

        uuid = "GPU-" + str(torch.cuda.get_device_properties(cuda_index).uuid)
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) != 0:
            raise RuntimeError("NVML handle lookup failed")
        self.get_reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.samples = []
        self.stop_flag = threading.Event()

    def _clock(self, fn, kind):
        v = self.ct.c_uint()
        return v.value if fn(self.h, kind, self.ct.byref(v)) == 0 else None

    def _run(self):
        r = self.ct.c_ulonglong()
        while not self.stop_flag.is_set():
            sm = self._clock(self.lib.nvmlDeviceGetClockInfo, 1)  # NVML_CLOCK_SM
            rs = r.value if self.get_reasons(self.h, self.ct.byref(r)) == 0 else 0
            if sm is not None:
                self.samples.append((sm, rs))
            time.sleep(0.002)

    def start(self):
        self.smax = self._clock(self.lib.nvmlDeviceGetMaxClockInfo, 1)
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def stop(self):
        self.stop_flag.set()
        self.thread.join(timeout=5)
        reasons = sorted({n for n, b in self.BITS.items() for _, rs in self.samples if rs & b})
        sm = [s for s, _ in self.samples]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.smax, "reasons": reasons,
                "samples": len(sm), "source": "nvml"}


class ClockSampler:
    """Clock / throttle-reason samples during the timed region: NVML polled
    every ~2 ms where libnvidia-ml loads, else nvidia-smi every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.nvml = None
        self.lines = []

    def start(self):
        try:
            self.nvml = _NvmlSampler(self.gpu)
            self.nvml.start()
            return
        except Exception:
            self.nvml = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            return self.nvml.stop()
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi"}


def _workload(n=N_LATTICE, kind="vortex"):
    from paper_2102_12933_gb300 import inputs

    if kind == "hybrid":
        # half of the lattice quads kept as quadrilaterals (with their two
        # artificial diagonals), half split into triangles
        mesh = inputs.hybrid_lattice(n, seed=1008, tri_fraction=0.5)
        return mesh, inputs.isentropic_vortex(mesh.xy)
    mesh, w0 = inputs.vortex_case(n, seed=1002)
    return mesh, w0


def vortex_config(n: int = N_LATTICE, parallelism: str = "single GPU") -> dict:
    """The `config` of the default line (shared by both arms)."""
    return {
        "workload": f"periodic isentropic vortex (beta=5, centre (5,5)) on a {n}x{n} jittered random-diagonal "
                    "torus lattice of [0,10]^2; two-level divergence stencils, degree-2 least squares, NU-WENO5, "
                    "SSP-RK3, CFL 0.5; one step = 3 stages",
        "nv": n * n, "ne": 3 * n * n, "stages_per_step": 3,
        "l2": "inputs larger than L2 (the edge and divergence tables streamed every stage exceed the 129 MB L2)",
        "parallelism": parallelism,
    }


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world_size: int, seconds: float) -> float:
    """Whole-job throughput of independent replicas: all ranks' units / the max time."""
    return world_size * units_per_rank / seconds


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def time_oracle(steps: int = 0, n_sample: int = 250, budget_s: float = 15.0, warmup: int = 0):
    """The FP64 oracle, as it stands, on the vortex workload family: SSP-RK3
    steps on an n_sample x n_sample mesh of the same family (one host core),
    after `warmup` untimed steps.  steps = 0 runs steps until `budget_s`
    seconds have passed (at most 200).  Returns (Mvertex/s, seconds, sample
    text, vertices)."""
    import oracle
    from paper_2102_12933_gb300 import inputs

    mesh, w = inputs.vortex_case(n_sample, seed=1002)
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.Lx, mesh.Ly)
    om.build_weights()
    dt = om.max_dt(w, CFL)
    for _ in range(warmup):
        w = om.rk3_step(w, dt)
    t0 = time.perf_counter()
    done = 0
    while (steps and done < steps) or (not steps and time.perf_counter() - t0 < budget_s and done < 200):
        w = om.rk3_step(w, dt)
        done += 1
    steps = done
    el = time.perf_counter() - t0
    value = mesh.nv * 3 * steps / el / 1e6
    sample = (f"{steps} SSP-RK3 step(s) of the single-threaded FP64 oracle on a {mesh.nv}-vertex mesh of the "
              f"same family (jittered random-diagonal torus, vortex, two-level degree-2 stencils)"
              + (f", after {warmup} untimed step(s)" if warmup else ""))
    return value, el, sample, int(mesh.nv)


def run_reference(args):
    """The oracle on this line's own workload (the full mesh of `--n`):
    `--warmup` untimed steps, then `--steps` timed SSP-RK3 steps."""
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    value, el, sample, nv = time_oracle(args.steps, n_sample=args.n, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Mvertex/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * el / max(args.steps, 1), 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": vortex_config(args.n, "replicas" if args.gpus > 1 else "single GPU"),
        "cpu_baseline": {"value": round(value, 4), "unit": "Mvertex/s", "cores": 1, "kind": "oracle",
                         "sample": sample, "nv": nv},
        "e2e": {"value": round(value, 4), "unit": "Mvertex/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_2102_12933_gb300 import fdu

    ws_, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if ws_ > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    hybrid = args.workload == "hybrid"
    mesh, w0 = _workload(args.n, args.workload)
    t_build = time.perf_counter()
    M = fdu.Mesh(mesh.xy, mesh.tri, mesh.Lx, mesh.Ly, device=local, **({"artificial_edges": 1} if hybrid else {}))
    t_build = time.perf_counter() - t_build
    info = M.info()
    nv, ne = M.nv, M.ne
    M.set_state(w0)
    dt = M.max_dt(CFL)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed_steps(prec, k, mesh_=None):
        mesh_ = M if mesh_ is None else mesh_
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(k):
            mesh_.rk_step(dt, prec, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(ev0.elapsed_time(ev1), dist)

    # ---------------- FP64 (headline)
    for _ in range(args.warmup):
        M.rk_step(dt, 64, stream=stream)
    M.profile(True)
    M.profile_read("edge", 64)
    M.profile_read("div", 64)
    sampler = ClockSampler(local)
    sampler.start()
    ms64 = timed_steps(64, args.steps)
    clocks = sampler.stop()
    edge_ms, edge_n = M.profile_read("edge", 64)
    div_ms, div_n = M.profile_read("div", 64)
    M.profile(False)
    w64 = M.get_state()

    # ---------------- precision 48 (FP64 state, double-word edge increments), same steps from w0
    M.set_state(w0)
    for _ in range(args.warmup):
        M.rk_step(dt, 48, stream=stream)
    M.set_state(w0)
    M.profile(True)
    M.profile_read("edge", 48)
    M.profile_read("div", 48)
    ms48 = timed_steps(48, args.steps)
    e48_ms, e48_n = M.profile_read("edge", 48)
    d48_ms, d48_n = M.profile_read("div", 48)
    M.profile(False)
    M.set_state(w0)
    res_diff48 = _rel_l2(M.residual(48), M.residual(64))

    # ---------------- FP32 residual path (FP64 accumulation), same steps from w0
    M.set_state(w0)
    for _ in range(args.warmup):
        M.rk_step(dt, 32, stream=stream)
    M.set_state(w0)
    M.profile(True)
    M.profile_read("edge", 32)
    M.profile_read("div", 32)
    ms32 = timed_steps(32, args.warmup + args.steps)
    e32_ms, e32_n = M.profile_read("edge", 32)
    d32_ms, d32_n = M.profile_read("div", 32)
    M.profile(False)
    w32 = M.get_state()
    # FP32 error against FP64 after 100 steps from the same initial state
    # (relative L2 of density and energy, the stated error of the FP32 form)
    err_steps = 100
    M.set_state(w0)
    M.rk_steps(dt, err_steps, 64, stream=stream)
    w64b = M.get_state()
    M.set_state(w0)
    M.rk_steps(dt, err_steps, 32, stream=stream)
    w32b = M.get_state()
    err32 = {"rho": _rel_l2(w32b[:, 0], w64b[:, 0]), "rhoE": _rel_l2(w32b[:, 3], w64b[:, 3]),
             "steps": err_steps}
    M.set_state(w0)
    M.rk_steps(dt, err_steps, 48, stream=stream)
    w48b = M.get_state()
    err48 = {"rho": _rel_l2(w48b[:, 0], w64b[:, 0]), "rhoE": _rel_l2(w48b[:, 3], w64b[:, 3]),
             "steps": err_steps}

    # ---------------- FP32 with the compact coefficient form: a second mesh
    # with f32_coef = 1 (NU-WENO5 values formed in FP32 in the edge kernel from
    # the FP64-built stencil gaps instead of streaming the FP64-built block),
    # the same steps from w0 and the same FP64 reference
    Mc = fdu.Mesh(mesh.xy, mesh.tri, mesh.Lx, mesh.Ly, device=local, f32_coef=1,
                  **({"artificial_edges": 1} if hybrid else {}))
    Mc.set_state(w0)
    for _ in range(args.warmup):
        Mc.rk_step(dt, 32, stream=stream)
    Mc.set_state(w0)
    Mc.profile(True)
    Mc.profile_read("edge", 32)
    msc = timed_steps(32, args.warmup + args.steps, Mc)
    ec_ms, ec_n = Mc.profile_read("edge", 32)
    Mc.profile(False)
    Mc.set_state(w0)
    Mc.rk_steps(dt, err_steps, 32, stream=stream)
    wcb = Mc.get_state()
    errc = {"rho": _rel_l2(wcb[:, 0], w64b[:, 0]), "rhoE": _rel_l2(wcb[:, 3], w64b[:, 3]), "steps": err_steps}
    Mc.close()

    # ---------------- end to end through the C-ABI with host buffers
    # pinned host buffers: the copies are DMA transfers of the caller's rows
    host_in = torch.from_numpy(np.ascontiguousarray(w0)).pin_memory().numpy()
    host_out = torch.zeros(w0.shape, dtype=torch.float64).pin_memory().numpy()
    # wall-clock over host round trips (each step's set_state and get_state
    # synchronise with the host): warm-up iterations first, then three blocks
    # of at least 50 timed steps each; the median block's time is reported, so
    # that a host-side hiccup in one block does not set the figure
    e2e_steps = max(50, args.steps)
    e2e_blocks = 3

    def e2e_block(prec):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            M.set_state(host_in)  # H2D of the step's input, checked and permuted to the internal order on the device
            M.rk_step(dt, prec)
            M.get_state(out=host_out)  # D2H of the step's result (synchronises)
        return max_over_ranks(time.perf_counter() - t0, dist)

    e2e_times = {}
    for prec in (64, 48):
        for _ in range(args.warmup):
            M.set_state(host_in)
            M.rk_step(dt, prec)
            M.get_state(out=host_out)
        e2e_times[prec] = sorted(e2e_block(prec) for _ in range(e2e_blocks))
    e2e_s = e2e_times[64][e2e_blocks // 2]
    e2e48_s = e2e_times[48][e2e_blocks // 2]

    # ---------------- figures
    stages = 3
    value = replica_throughput(nv * stages * args.steps, ws_, ms64 / 1e3) / 1e6
    value32 = replica_throughput(nv * stages * (args.warmup + args.steps), ws_, ms32 / 1e3) / 1e6
    value48 = replica_throughput(nv * stages * args.steps, ws_, ms48 / 1e3) / 1e6
    e48_avg_ms = e48_ms / max(e48_n, 1)
    tf48 = FLOP_EDGE64 * ne / (e48_avg_ms / 1e3) / 1e12
    e2e_value = replica_throughput(nv * stages * e2e_steps, ws_, e2e_s) / 1e6
    e32_avg = e32_ms / max(e32_n, 1)
    d32_avg = d32_ms / max(d32_n, 1)
    stage32_ms = ms32 / (stages * (args.warmup + args.steps))
    edge_avg_ms = edge_ms / max(edge_n, 1)
    div_avg_ms = div_ms / max(div_n, 1)
    achieved_tf = FLOP_EDGE64 * ne / (edge_avg_ms / 1e3) / 1e12
    fp64_probe = fdu.probe_fma(local, 64)
    peaks = _peaks()
    vnnz, ennz = info["div_vert_nnz"], info["div_edge_nnz"]
    div_flops = FLOP_DIV64_PER_VENTRY * vnnz + FLOP_DIV64_PER_EENTRY * ennz + FLOP_DIV64_FIXED * nv
    # FP32 kernels are HBM-bound.  Bytes per launch of the kernels' own tables:
    edge32_bytes = ne * (24 + 26 * 4 + 16) + nv * 16  # ids, 24 coefficients and the normal, flux; FP32 state once
    edge32c_bytes = ne * (24 + 4 * 4 + 8 + 16) + nv * 16  # compact form: ids, 4 stencil gaps, normal, flux
    div32_bytes = (vnnz * 12 + ennz * 8 + nv * 8) + nv * (32 + 32 + 32 + 32 + 16) + ne * 16 + nv * 32
    # and the method's algorithmic bytes at p = 4 (compact edge form: 6 ids, 4
    # curve coordinates and n per edge; divergence tables (2J+K+2) p + 4 (J+K)
    # per vertex, J and K this mesh's entry counts), counted once each:
    p32 = 4
    edge32_alg = ne * (24 + 6 * p32 + 4 * p32) + nv * 4 * p32  # ids + edge data, flux write; state read
    div32_alg = ((2 * vnnz + ennz + 2 * nv) * p32 + 4 * (vnnz + ennz)) + ne * 4 * p32 + nv * 4 * p32 \
        + nv * (64 + 16)  # tables, flux read, residual write, stage (FP64 w_n in / w_new out, FP32 copy)
    hbm = peaks.get("hbm_gbs", 6800.0)
    fp32_probe = fdu.probe_fma(local, 32)  # TFLOP/s, FMA = 2 flop
    fp32_issue_peak = fp32_probe / 2 * 1e12  # thread instructions per second on the FMA pipe
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "Mvertex/s",
        "n_gpus": ws_,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms64 / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": vortex_config(args.n, "replicas" if ws_ > 1 else "single GPU"),
        "roofline": {
            "kernel": "edge_flux_f64",
            "bound": "alu",
            "achieved": round(achieved_tf, 4),
            "peak": FP64_PEAK_NOMINAL_TFLOPS,
            "unit": "TFLOP/s",
            "frac": round(achieved_tf / FP64_PEAK_NOMINAL_TFLOPS, 4),
            "traffic": (round(TRAFFIC_EDGE64_B_PER_EDGE * ne) if TRAFFIC_EDGE64_B_PER_EDGE else None),
            "traffic_unit": "bytes per launch",
            "peak_source": "nominal GB300 FP64 rate (no FP64 figure in MEASURED_PEAKS.json)",
            "peak_probe": round(fp64_probe, 4),
            "frac_of_probe": round(achieved_tf / fp64_probe, 4),
            "flop_per_edge": FLOP_EDGE64,
            "ncu_fp64_pipe_busy": NCU_EDGE64_FP64_PIPE_BUSY,
            "ncu_fp64_instr_per_edge": NCU_EDGE64_FP64_INSTR_PER_EDGE,
            "avg_launch_ms": round(edge_avg_ms, 4),
            "share_of_step": round(edge_ms / ms64, 4) if ms64 > 0 else None,
            "div_kernel": {"avg_launch_ms": round(div_avg_ms, 4),
                           "achieved_tflops": round(div_flops / (div_avg_ms / 1e3) / 1e12, 4)},
        },
        "f64_dw": {
            "precision": 48,
            "value": round(value48, 3), "unit": "Mvertex/s", "ms_per_step": round(ms48 / args.steps, 4),
            "speedup_vs_f64": round(value48 / value, 3),
            "dtype": "f64 state, divergence and state-sized flux terms; edge-flux increments in f32x2 double words",
            "residual_vs_f64": res_diff48,
            "error_vs_f64": err48,
            "edge_kernel": {"kernel": "edge_flux_dw", "bound": "alu (FP32 issue)",
                            "avg_launch_ms": round(e48_avg_ms, 4),
                            "fp64_equivalent_tflops": round(tf48, 4),
                            "thread_instr_per_s": round(NCU_EDGE48_THREAD_INSTR_PER_EDGE * ne / (e48_avg_ms / 1e3)),
                            "peak_thread_instr_per_s": round(fp32_issue_peak),
                            "peak_source": "fdu_probe_fma(32) measured live: FP32 FMA chains, one thread "
                                           "instruction per FMA",
                            "frac_of_fp32_issue": round(NCU_EDGE48_THREAD_INSTR_PER_EDGE * ne / (e48_avg_ms / 1e3)
                                                        / fp32_issue_peak, 4),
                            "ncu_issue_active": NCU_EDGE48_ISSUE_ACTIVE, "ncu_fma_pipe": NCU_EDGE48_FMA_PIPE,
                            "ncu_fp64_pipe": NCU_EDGE48_FP64_PIPE,
                            "ncu_thread_instr_per_edge": round(NCU_EDGE48_THREAD_INSTR_PER_EDGE),
                            "traffic": round(TRAFFIC_EDGE48_B_PER_EDGE * ne), "traffic_unit": "bytes per launch"},
            "div_kernel": {"avg_launch_ms": round(d48_ms / max(d48_n, 1), 4)},
            "e2e": {"value": round(replica_throughput(nv * stages * e2e_steps, ws_, e2e48_s) / 1e6, 3),
                    "unit": "Mvertex/s", "h2d_bytes_per_step": nv * 32, "d2h_bytes_per_step": nv * 32,
                    "steps": e2e_steps, "blocks": e2e_blocks, "statistic": "median block",
                    "block_values": [round(replica_throughput(nv * stages * e2e_steps, ws_, t) / 1e6, 3)
                                     for t in e2e_times[48]]},
        },
        "fp32": {
            "value": round(value32, 3), "unit": "Mvertex/s", "speedup_vs_f64": round(value32 / value, 3),
            "error_vs_f64": err32,
            "coefficients": "NU-WENO5 block built in FP64 on the host, streamed rounded to FP32 (104 B per edge)",
            "edge_kernel": {"avg_launch_ms": round(e32_avg, 4),
                            "bound": "coefficient stream and gather latency (neither DRAM nor issue saturated)",
                            "ncu_issue_active": NCU_EDGE32_ISSUE_ACTIVE, "ncu_fma_pipe": NCU_EDGE32_FMA_PIPE,
                            "ncu_dram_throughput": NCU_EDGE32_DRAM,
                            "traffic": (round(TRAFFIC_EDGE32_B_PER_EDGE * ne) if TRAFFIC_EDGE32_B_PER_EDGE else None),
                            "traffic_unit": "bytes per launch",
                            "achieved_gbs": round(edge32_bytes / (e32_avg / 1e3) / 1e9, 1),
                            "frac_hbm": round(edge32_bytes / (e32_avg / 1e3) / 1e9 / hbm, 4),
                            "algorithmic_bytes": int(edge32_alg),
                            "frac_hbm_algorithmic": round(edge32_alg / (e32_avg / 1e3) / 1e9 / hbm, 4)},
            "div_kernel": {"avg_launch_ms": round(d32_avg, 4),
                           "achieved_gbs": round(div32_bytes / (d32_avg / 1e3) / 1e9, 1),
                           "frac_hbm": round(div32_bytes / (d32_avg / 1e3) / 1e9 / hbm, 4),
                           "algorithmic_bytes": int(div32_alg),
                           "frac_hbm_algorithmic": round(div32_alg / (d32_avg / 1e3) / 1e9 / hbm, 4)},
            "stage": {"avg_ms": round(stage32_ms, 4), "algorithmic_bytes": int(edge32_alg + div32_alg),
                      "frac_hbm_algorithmic": round((edge32_alg + div32_alg) / (stage32_ms / 1e3) / 1e9 / hbm, 4)},
            "frac_hbm_note": "frac_hbm divides the kernel's own table bytes; frac_hbm_algorithmic the method's "
                             "compact bytes (edge: 64 B per edge + 16 B per vertex, which the compact "
                             "coefficient form's tables are; divergence: its stencil tables, flux read, "
                             "residual write and the stage's 80 B per vertex)",
            "compact_coefficients": {
                "note": "mesh option f32_coef = 1: NU-WENO5 values formed in FP32 in the edge kernel from the "
                        "stencil gaps (built in FP64 on the host) instead of the streamed FP64-built block; "
                        "same mesh, initial state, steps and FP64 reference",
                "value": round(replica_throughput(nv * stages * (args.warmup + args.steps), ws_, msc / 1e3) / 1e6, 3),
                "unit": "Mvertex/s", "error_vs_f64": errc,
                "edge_kernel": {"avg_launch_ms": round(ec_ms / max(ec_n, 1), 4),
                                "bound": "FP32 issue",
                                "ncu_issue_active": NCU_EDGE32G_ISSUE_ACTIVE, "ncu_fma_pipe": NCU_EDGE32G_FMA_PIPE,
                                "ncu_dram_throughput": NCU_EDGE32G_DRAM,
                                "traffic": round(TRAFFIC_EDGE32G_B_PER_EDGE * ne), "traffic_unit": "bytes per launch",
                                "frac_hbm_algorithmic": round(edge32c_bytes / (ec_ms / max(ec_n, 1) / 1e3) / 1e9 / hbm,
                                                              4)},
            },
        },
        "e2e": {"value": round(e2e_value, 3), "unit": "Mvertex/s", "h2d_bytes_per_step": nv * 32,
                "d2h_bytes_per_step": nv * 32, "steps": e2e_steps, "blocks": e2e_blocks, "statistic": "median block",
                "block_values": [round(replica_throughput(nv * stages * e2e_steps, ws_, t) / 1e6, 3)
                                 for t in e2e_times[64]]},
        "gpu_launches": 6 * args.steps,
        "clocks": clocks,
    }
    if hybrid:
        line["config"].update(
            workload=f"periodic isentropic vortex on a {args.n}x{args.n} jittered hybrid torus lattice of [0,10]^2: "
                     "half of the quads kept as quadrilaterals with both artificial diagonals (Section 2.2.2), half "
                     "split into triangles; two-level stencils, degree-2 least squares, NU-WENO5, SSP-RK3, CFL 0.5",
            ne=int(ne), cells=int(mesh.nt))
    if not hybrid and not args.skip_legs:
        # config 5 (adjoint, 250k vertices, FP64): timing with the paper's eps;
        # the FD check with a smooth eps (32 directions for the FP64 adjoint,
        # 8 for the precision-48 adjoint; steps 1e-5, 1e-6, 1e-7: at eps =
        # 1e-6 steps of 1e-4 and above leave the weights' linear range)
        line["adjoint"] = adjoint_figures(args.n, local, (("eps_1e-40", 1e-40, 0, 0, ()),
                                                          ("eps_1e-6", 1e-6, 32, 8, (1e-5, 1e-6, 1e-7))))
        # config 4 (64 meshes, one persistent launch per stage)
        line["batch"] = batch_figures(args.steps, args.warmup, local)
        line["gpu_launches_note"] = ("gpu_launches counts the headline's timed FP64 steps; the adjoint and batch "
                                     "sub-objects are timed in their own regions")
    if rank == 0 and not args.no_cpu_baseline and not hybrid:
        v, el, sample, nv_s = time_oracle()
        line["cpu_baseline"] = {"value": round(v, 4), "unit": "Mvertex/s", "cores": 1, "kind": "oracle",
                                "sample": sample, "nv": nv_s, "seconds": round(el, 2)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    M.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _advance_both(M, w0, real, t_end, max_steps, err_steps=16):
    """FP64, precision-48 and FP32 adaptive runs from w0 to t_end (at most
    max_steps steps), wall-clock timed between the host's time checks every
    8 steps; the other states are compared with the FP64 one after
    err_steps steps."""
    import torch

    from paper_2102_12933_gb300 import fdu

    n_real = int(real.sum())
    out, states = {}, {}
    for prec in (64, 48, 32):
        M.set_state(w0)
        M.advance(0.5, t_end, prec, max_steps=8)  # warm-up (graph capture)
        M.set_state(w0)
        M.fallback_count(reset=True)
        M.limited_count(reset=True)
        steps, t, el, status = 0, 0.0, 0.0, "reached t_end"
        while t < t_end and steps < max_steps:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                k, t = M.advance(0.5, t_end, prec, max_steps=8)
            except fdu.FduError as e:
                status = f"stopped: {e}"
                break
            torch.cuda.synchronize()
            el += time.perf_counter() - t0
            steps += k
            if steps == err_steps:
                states[prec] = M.get_state()
        if t < t_end and status == "reached t_end":
            status = f"stopped at max_steps={max_steps}"
        out[prec] = {"steps": steps, "t": t, "seconds": round(el, 3), "status": status,
                     "value": round(n_real * 3 * steps / el / 1e6, 2) if el > 0 else None,
                     "fallback_edges": M.fallback_count(), "safeguarded_vertex_stages": M.limited_count()}
    err = {}
    for prec in (48, 32):
        if 64 in states and prec in states:
            err[prec] = {"rho": _rel_l2(states[prec][real, 0], states[64][real, 0]),
                         "rhoE": _rel_l2(states[prec][real, 3], states[64][real, 3]), "steps": err_steps}
    return out, err


def _ghost_line(out, err, workload, t_build):
    return {
        "metric": METRIC, "value": out[64]["value"], "unit": "Mvertex/s", "n_gpus": 1,
        "steps": out[64]["steps"], "warmup": 1,
        "ms_per_step": round(1e3 * out[64]["seconds"] / max(out[64]["steps"], 1), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "host_build_s": round(t_build, 2)},
        "fp64": out[64],
        "f64_dw": dict(out[48], speedup_vs_f64=(round(out[48]["value"] / out[64]["value"], 3)
                                                if out[48]["value"] and out[64]["value"] else None),
                       error_vs_f64=err.get(48)),
        "fp32": dict(out[32], speedup_vs_f64=(round(out[32]["value"] / out[64]["value"], 3)
                                              if out[32]["value"] and out[64]["value"] else None),
                     error_vs_f64=err.get(32)),
    }


def run_riemann(args):
    """Config 3: four-quadrant 2D Riemann problem on [0,1]^2, ~1M vertices
    (1000 x 1000 jittered lattice + 5 transmissive ghost layers), advanced to
    t = 0.3 with the device-computed CFL time step, in FP64 and FP32."""
    import torch

    from paper_2102_12933_gb300 import fdu, inputs

    ws_, rank, local = _dist()
    torch.cuda.set_device(local)
    n = args.n if args.n != N_LATTICE else 1000
    mesh, w0 = inputs.riemann_case(n, ghost_layers=5, seed=1003)
    t_build = time.perf_counter()
    # the unguarded method turns non-physical on this problem; the stage
    # positivity safeguard keeps rho, p > 0 so the run reaches t_end
    M = fdu.Mesh(mesh.xy, mesh.tri, 0.0, 0.0, device=local, ghost_donor=mesh.ghost_donor, positivity_alpha=0.1)
    t_build = time.perf_counter() - t_build
    real = mesh.ghost_donor < 0
    out, err = _advance_both(M, w0, real, args.t_end, args.riemann_max_steps)
    line = _ghost_line(out, err, f"four-quadrant 2D Riemann problem on [0,1]^2, {n}x{n} jittered lattice + 5 "
                                 f"transmissive ghost layers ({mesh.nv} vertices, {int(real.sum())} real), to t = "
                                 f"{args.t_end} with device-side CFL 0.5 time steps and the stage positivity safeguard "
                                 "(alpha 0.1) (wall-clock timed, includes the host's time checks every 8 steps)",
                       t_build)
    print(json.dumps(line), flush=True)
    M.close()
    return 0


def run_shock_vortex(args):
    """Shock-vortex interaction (Section 3.2): Mach 1.2 stationary shock at
    x = 0 and the M_v = 1 isentropic vortex at (4, 0) on [-65, 15] x [-40,
    40], periodic in y, Dirichlet ghost columns in x; regular diagonalised
    lattice at the paper's finest spacing 0.08 (n = 1000 across y), with CFL
    0.5 and the stage positivity safeguard, FP64 and FP32.  By default to
    t = 3, while the vortex approaches the shock: at this spacing its
    passage through the shock (t ~ 3.3) drives the core towards vacuum and
    the CFL step collapses; with --n 320 (h = 0.25) the run goes through the
    interaction (--t-end 16)."""
    import torch

    from paper_2102_12933_gb300 import fdu, inputs

    ws_, rank, local = _dist()
    torch.cuda.set_device(local)
    n = args.n if args.n != N_LATTICE else 1000
    mesh, w0 = inputs.shock_vortex_case(n)
    t_build = time.perf_counter()
    # the paper's M_v = 1 vortex turns the unguarded method non-physical
    # within t < 1 on these lattices; the safeguard keeps rho, p > 0
    M = fdu.Mesh(mesh.xy, mesh.tri, 0.0, 80.0, device=local, ghost_donor=mesh.ghost_donor, positivity_alpha=0.1)
    t_build = time.perf_counter() - t_build
    real = mesh.ghost_donor < 0
    t_end = args.t_end if args.t_end != 0.3 else 3.0
    out, err = _advance_both(M, w0, real, t_end, args.riemann_max_steps if args.riemann_max_steps != 400 else 4000)
    line = _ghost_line(out, err, f"shock-vortex interaction (Section 3.2) on [-65,15]x[-40,40], periodic in y, "
                                 f"{n} points across y (h = {80.0 / n:g}), regular diagonalised lattice + 5 Dirichlet "
                                 f"ghost columns per side ({mesh.nv} vertices, {int(real.sum())} real), Mach 1.2 shock, "
                                 f"M_v = 1 vortex at (4, 0), to t = {t_end} with device-side CFL 0.5 time steps and the "
                                 "stage positivity safeguard (alpha 0.1) (wall-clock timed)", t_build)
    print(json.dumps(line), flush=True)
    M.close()
    return 0


def batch_figures(steps, warmup, local, err_steps=100):
    """Config 4: 64 independent periodic vortex meshes, sizes log-uniform in
    5k..200k vertices, strengths in [1,5], centres in [3,7]^2, each with its
    own CFL time step, advanced by one persistent launch per RK stage
    (CUDA-graph replays), launch shape picked by the autotuner; FP32
    residual with FP64 state accumulation, with the FP64 and precision-48
    residuals timed beside it.  Returns (figures, workload text, vertices)."""
    import torch

    from paper_2102_12933_gb300 import fdu, inputs

    n_i, beta, centres = inputs.batch_sizes(64, seed=2004)
    meshes, states = [], []
    for i in range(len(n_i)):
        m, w = inputs.vortex_case(int(n_i[i]), seed=3000 + i, beta=float(beta[i]), centre=tuple(centres[i]))
        meshes.append((m.xy, m.tri))
        states.append(w)
    w0 = np.concatenate(states)
    t_build = time.perf_counter()
    B = fdu.Batch(meshes, L=10.0, device=local)
    t_build = time.perf_counter() - t_build
    B.set_state(w0)
    dts = B.batch_max_dt(CFL)
    B.set_dt(dts)
    stream = torch.cuda.current_stream()
    res = {}
    for prec in (32, 64, 48):
        B.set_state(w0)
        t, b, ms_tune = B.autotune(prec)
        B.batch_rk_steps(warmup, prec, stream=stream)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        B.batch_rk_steps(steps, prec, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        res[prec] = {"value": round(B.nv * 3 * steps / (ms / 1e3) / 1e6, 2), "unit": "Mvertex/s",
                     "ms_per_step": round(ms / steps, 4),
                     "launch": {"threads": t, "blocks_per_sm": b, "autotune_ms_per_step": round(ms_tune, 4)}}
    # errors against FP64 after the same steps from the same state, over all meshes
    finals = {}
    for prec in (64, 48, 32):
        B.set_launch(res[prec]["launch"]["threads"], res[prec]["launch"]["blocks_per_sm"])  # its tuned shape
        B.set_state(w0)
        B.batch_rk_steps(err_steps, prec, stream=stream)
        finals[prec] = B.get_state()
    for prec in (48, 32):
        res[prec]["error_vs_f64"] = {"rho": _rel_l2(finals[prec][:, 0], finals[64][:, 0]),
                                     "rhoE": _rel_l2(finals[prec][:, 3], finals[64][:, 3]), "steps": err_steps}
    workload = (f"{len(n_i)} periodic vortex meshes, {int(B.nv)} vertices in total (sizes {int(np.min(n_i) ** 2)}.."
                f"{int(np.max(n_i) ** 2)}), per-mesh CFL 0.5 time steps, one persistent launch per RK stage, "
                "CUDA-graph replays, autotuned launch shape")
    out = {"workload": workload, "nv": int(B.nv), "host_build_s": round(t_build, 2), "steps": steps,
           "fp32": res[32], "fp64": res[64],
           "f64_dw": dict(res[48], speedup_vs_f64=round(res[48]["value"] / res[64]["value"], 3)),
           "gpu_launches_per_step": 3}
    B.close()
    return out


def run_batch(args):
    """Config 4 as its own line (see batch_figures)."""
    import torch

    ws_, rank, local = _dist()
    torch.cuda.set_device(local)
    b = batch_figures(args.steps, args.warmup, local)
    line = {
        "metric": METRIC, "value": b["fp32"]["value"], "unit": "Mvertex/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["fp32"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 residual, f64 accumulation", "data": "synthetic",
        "config": {"workload": b["workload"], "host_build_s": b["host_build_s"]},
        "fp32": b["fp32"], "fp64": b["fp64"], "f64_dw": b["f64_dw"],
    }
    print(json.dumps(line), flush=True)
    return 0


def _fd_check(J, g, d_gen, shape, n_dirs, steps_h):
    """Best relative error per direction of <g, d> against central
    differences of J (2nd and 4th order) on the step ladder steps_h."""
    import torch

    errs = []
    for _ in range(n_dirs):
        d = torch.randn(shape, generator=d_gen, device="cuda", dtype=torch.float64)
        a = float((g * d).sum())
        best = None
        for h in steps_h:
            jp, jm = J(h * d), J(-h * d)
            jp2, jm2 = J(2 * h * d), J(-2 * h * d)
            for fd in ((jp - jm) / (2 * h), (8 * (jp - jm) - (jp2 - jm2)) / (12 * h)):
                e = abs(fd - a) / abs(a)
                best = e if best is None else min(best, e)
        errs.append(best)
    return errs


def adjoint_figures(n, local, legs, n_steps=50, k=10):
    """Config 5: gradient of J = 1/2 sum_v (rho_v(T) - rho_exact,v(T))^2 after
    n_steps SSP-RK3 steps of the 250k-vertex vortex with respect to the
    initial state, by the hand-written adjoint with a checkpoint every k
    steps, timed against the forward pass, and checked against central
    differences on seeded N(0,1) directions over all 4V initial components.
    `legs` lists (label, weno eps, FD directions for the FP64 adjoint, FD
    directions for the precision-48 adjoint, FD step ladder).  Where the
    smoothness indicators sit at rounding level (the near-uniform far field
    with the paper's eps = 1e-40) the weights are not differentiable at the
    FD step's scale, so the FD check belongs to a smooth eps."""
    import torch

    from paper_2102_12933_gb300 import fdu, inputs

    mesh, w0 = inputs.vortex_case(n, seed=1005)
    stream = torch.cuda.current_stream()
    w0d = torch.tensor(w0, device="cuda")

    def timed(fn, reps):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    result = {}
    for label, eps, fd_dirs, fd_dirs48, steps_h in legs:
        M = fdu.Mesh(mesh.xy, mesh.tri, mesh.Lx, mesh.Ly, device=local, weno_eps=eps)
        M.set_state(w0d)
        dt = M.max_dt(CFL)
        ex = torch.tensor(inputs.isentropic_vortex(mesh.xy, t=n_steps * dt)[:, 0], device="cuda")
        wT = torch.empty_like(w0d)

        def J_and_lam(w):
            M.set_state(w)
            M.rk_steps(dt, n_steps, 64, stream=stream)
            M.get_state(out=wT)
            r = wT[:, 0] - ex
            lam = torch.zeros_like(wT)
            lam[:, 0] = r
            return 0.5 * float((r * r).sum()), lam

        out = torch.empty_like(w0d)
        M.set_state(w0d)
        t_res = timed(lambda: M.residual(64, out=out, stream=stream), 20)
        lam_r = torch.randn_like(w0d)
        t_vjp = timed(lambda: M.residual_vjp(lam_r, out=out, stream=stream), 20)
        t_fwd = timed(lambda: (M.set_state(w0d, stream=stream), M.rk_steps(dt, n_steps, 64, stream=stream)), 3)
        J0, lamT = J_and_lam(w0d)
        grad = torch.empty_like(w0d)

        def adj():
            M.set_state(w0d, stream=stream)
            M.adjoint_rk(dt, n_steps, lamT, out=grad, checkpoint_every=k, stream=stream)

        t_adj = timed(adj, 3)
        g = grad.clone()
        # the same gradient with one segment (every stage state kept, 3 x 50
        # states of 8 MB: no recomputation)
        grad1 = torch.empty_like(w0d)

        def adj1():
            M.set_state(w0d, stream=stream)
            M.adjoint_rk(dt, n_steps, lamT, out=grad1, checkpoint_every=n_steps, stream=stream)

        t_adj1 = timed(adj1, 3)
        one_seg = {"adjoint_ms": round(t_adj1, 3), "adjoint_over_forward": round(t_adj1 / t_fwd, 3),
                   "max_abs_diff_vs_checkpointed": float((grad1 - g).abs().max())}
        J = lambda dw: J_and_lam(w0d + dw)[0]  # noqa: E731
        fd = None
        if fd_dirs:
            errs = _fd_check(J, g, torch.Generator(device="cuda").manual_seed(5005), w0d.shape, fd_dirs, steps_h)
            fd = {"directions": fd_dirs, "steps_h": list(steps_h),
                  "differences": "central, 2nd and 4th order; best per direction",
                  "max_rel_err": float(np.max(errs)), "median_rel_err": float(np.median(errs)),
                  "within_1e-6": int(np.sum(np.array(errs) <= 1e-6))}
        # the same with the double-word edge-flux VJP (adjoint precision 48)
        M.set_adjoint_precision(48)
        M.set_state(w0d)
        t_vjp48 = timed(lambda: M.residual_vjp(lam_r, out=out, stream=stream), 20)
        t_adj48 = timed(adj, 3)
        g48 = grad.clone()
        fd48 = None
        if fd_dirs48:
            errs48 = _fd_check(J, g48, torch.Generator(device="cuda").manual_seed(5005), w0d.shape, fd_dirs48,
                               steps_h)
            fd48 = {"directions": fd_dirs48, "steps_h": list(steps_h), "max_rel_err": float(np.max(errs48)),
                    "median_rel_err": float(np.median(errs48)),
                    "within_1e-6": int(np.sum(np.array(errs48) <= 1e-6))}
        M.set_adjoint_precision(64)
        t_fwd48 = timed(lambda: (M.set_state(w0d, stream=stream), M.rk_steps(dt, n_steps, 48, stream=stream)), 3)
        adjoint48 = {"residual_vjp_ms": round(t_vjp48, 4), "residual_vjp_over_residual": round(t_vjp48 / t_res, 3),
                     "adjoint_ms": round(t_adj48, 3), "adjoint_over_forward": round(t_adj48 / t_fwd, 3),
                     "forward48_ms": round(t_fwd48, 3), "adjoint_over_forward48": round(t_adj48 / t_fwd48, 3),
                     "note": "adjoint precision 48: double-word edge-flux VJP and precision-48 forward and "
                             "recomputed steps; adjoint_over_forward is against the FP64 forward",
                     "gradient_rel_diff_vs_f64": float((g48 - g).norm() / g.norm()), "fd_check": fd48}
        result[label] = {"weno_eps": eps, "residual_ms": round(t_res, 4), "residual_vjp_ms": round(t_vjp, 4),
                         "residual_vjp_over_residual": round(t_vjp / t_res, 3), "forward_ms": round(t_fwd, 3),
                         "adjoint_ms": round(t_adj, 3), "adjoint_over_forward": round(t_adj / t_fwd, 3),
                         "one_segment": one_seg, "J": J0, "fd_check": fd, "precision48_vjp": adjoint48}
        M.close()
    workload = (f"periodic vortex, {mesh.nv} vertices (jittered random-diagonal 500x500 torus lattice); J = 1/2 "
                f"sum (rho(T) - rho_exact(T))^2 after {n_steps} SSP-RK3 steps (CFL 0.5); adjoint with a "
                f"checkpoint every {k} steps; FP64")
    return {"workload": workload, "nv": int(mesh.nv), "n_steps": n_steps, "checkpoint_every": k, "legs": result}


def run_adjoint(args):
    """Config 5 as its own line: timing and FD checks for both eps (see
    adjoint_figures), 32 directions on the full step ladder."""
    import torch

    ws_, rank, local = _dist()
    torch.cuda.set_device(local)
    ladder = (1e-4, 1e-5, 1e-6, 1e-7)
    a = adjoint_figures(args.n, local, (("eps_1e-40", 1e-40, 32, 8, ladder), ("eps_1e-6", 1e-6, 32, 8, ladder)))
    main = a["legs"]["eps_1e-40"]
    line = {
        "metric": METRIC, "value": main["residual_vjp_over_residual"], "unit": "residual VJP / residual time",
        "n_gpus": 1, "steps": a["n_steps"], "warmup": 1, "ms_per_step": round(main["adjoint_ms"] / a["n_steps"], 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": a["workload"]},
        "adjoint": a["legs"],
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sod(args):
    """The paper's 2D Sod problem (Section 3.2) with its fifth-order setting:
    degree-5 least squares, periodic [-1,1]^2, regular diagonalised 55x55
    mesh (3025 points), device-side CFL 0.5 steps to t = 0.6, FP64, precision 48
    and FP32."""
    import torch

    from paper_2102_12933_gb300 import fdu, inputs

    ws_, rank, local = _dist()
    torch.cuda.set_device(local)
    mesh, w0 = inputs.sod_case(55)
    M = fdu.Mesh(mesh.xy, mesh.tri, 2.0, 2.0, lsq_degree=5, lsq_levels=2, device=local)
    out = {}
    states = {}
    for prec in (64, 48, 32):
        M.set_state(w0)
        M.advance(0.5, 0.6, prec, max_steps=8)
        M.set_state(w0)
        M.fallback_count(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps, t = M.advance(0.5, 0.6, prec)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        w = M.get_state()
        rho = w[:, 0]
        p = 0.4 * (w[:, 3] - 0.5 * (w[:, 1] ** 2 + w[:, 2] ** 2) / rho)
        out[prec] = {"steps": steps, "t": t, "seconds": round(el, 4),
                     "value": round(M.nv * 3 * steps / el / 1e6, 3), "fallback_edges": M.fallback_count(),
                     "rho_range": [float(rho.min()), float(rho.max())], "p_range": [float(p.min()), float(p.max())]}
        states[prec] = w
    line = {
        "metric": METRIC, "value": out[64]["value"], "unit": "Mvertex/s", "n_gpus": 1, "steps": out[64]["steps"],
        "warmup": 1, "ms_per_step": round(1e3 * out[64]["seconds"] / max(out[64]["steps"], 1), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "2D Sod problem (Section 3.2), periodic [-1,1]^2, regular diagonalised 55x55 mesh "
                               "(3025 points), degree-5 least squares on two-level stencils, CFL 0.5, to t = 0.6 "
                               "(wall-clock timed; a mesh this small is launch-bound)"},
        "fp64": out[64],
        "f64_dw": dict(out[48], error_vs_f64_rho=_rel_l2(states[48][:, 0], states[64][:, 0])),
        "fp32": dict(out[32], error_vs_f64_rho=_rel_l2(states[32][:, 0], states[64][:, 0])),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-legs", dest="skip_legs", action="store_true",
                    help="leave out the separately timed adjoint and batch sub-objects (for profiling the "
                         "headline's launches; the headline's timed work is the same)")
    ap.add_argument("--n", type=int, default=N_LATTICE, help="lattice size (n x n vertices); 500 = the workload")
    ap.add_argument("--workload", default="vortex", choices=["vortex", "riemann", "batch", "adjoint", "sod", "hybrid", "shock_vortex"],
                    help="vortex: the 250k periodic vortex (default line); riemann: the 1M-vertex "
                         "transmissive four-quadrant Riemann problem to t_end")
    ap.add_argument("--t-end", dest="t_end", type=float, default=0.3)
    ap.add_argument("--riemann-max-steps", dest="riemann_max_steps", type=int, default=400)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "riemann":
        return run_riemann(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "sod":
        return run_sod(args)
    if args.workload == "shock_vortex":
        return run_shock_vortex(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
