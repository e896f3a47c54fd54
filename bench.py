"""Throughput of the fused D2Q9 improved-MRT pseudopotential step on GB300.

Workload (one GPU): a 4096 x 4096 periodic FP32 field holding 64 non-overlapping
droplets (radii uniform in [40, 200], seed 5) of the Carnahan-Starling fluid with
a = 0.25, T = 0.6 T_c, sigma = 0.114, liquid/vapour viscosities 0.05/0.5 with the
relaxation time linear in rho.  A benchmark step is one time step of the whole field
(one launch of the fused kernel); every 100th step also runs the diagnostics pass
(mass, momentum, max |v|, |d rho|_inf).  The state (1.2 GB) is far larger than L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the host
cores instead (each step: one oracle step on a 1024 x 1024 window of the same field).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX = NY = 4096  # default grid; --grid changes it (smaller grids are for profiling only)
A, B, R = 0.25, 4.0, 1.0
TR = 0.6
SIGMA = 0.114
NU_L, NU_V = 0.05, 0.5
RATES = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)
DIAG_EVERY = 100
WARM_HORIZON = 60000  # steps each initialisation of the warm-start comparison runs
BYTES_PER_LU = 72  # 9 float populations read + 9 written per lattice update
PREC = "fp32"      # --precision: fp32 (deviation storage, the headline) or fp64 (parity mode)
FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64, nominal
REF_WINDOW = 1024
METRIC = "MLUPS (D2Q9 MRT-pseudopotential step, 4096^2, FP32)"


def n_droplets():
    return max(1, 64 * NX * NY // (4096 * 4096))


def workload_name():
    return "droplets%d_%dx%d_%s" % (n_droplets(), NX, NY, PREC)


def eos_T():
    from paper_1211_6932_gb300 import workloads as wl
    return TR * wl.t_crit(A, B, R)


def field(rho_l, rho_v, n=None, droplets=None):
    """The workload's density field: `droplets` non-overlapping droplets, radii uniform
    in [40, 200], on an n x n periodic lattice (seed 5)."""
    from paper_1211_6932_gb300 import workloads as wl
    n = NX if n is None else n
    droplets = n_droplets() if droplets is None else droplets
    rho, _, _ = wl.multi_droplets(n, n, rho_l, rho_v, 4.0, droplets, 40.0, 200.0, seed=5)
    return rho


def ref_field(rho_l, rho_v):
    """Bounded sample for the CPU oracle: the same recipe on a 1024^2 lattice with 4
    droplets (the same liquid fraction as 64 droplets on 4096^2)."""
    return field(rho_l, rho_v, n=REF_WINDOW, droplets=4)


def config(extra=None):
    c = {"workload": workload_name(), "grid": [NX, NY], "droplets": n_droplets(), "a": A,
         "T_over_Tc": TR,
         "sigma": SIGMA, "nu_l": NU_L, "nu_v": NU_V, "visc_mode": "linear",
         "diag_every": DIAG_EVERY,
         "l2": "state %.2f GB > 129 MB L2, no flush" % (2 * (36 if PREC == "fp32" else 72)
                                                         * NX * NY / 1e9),
         "parallelism": "replicas"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash(precision="fp32"):
    """Hash of the sources that define the step kernel of a precision."""
    h = hashlib.sha256()
    for f in ("lbm_device.cuh", "lbm_kernels_impl.cuh", "lbm_kernels_f%s.cu" % precision[2:]):
        with open(os.path.join(ROOT, "paper_1211_6932_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


GRAPH_STEPS = 64  # steps per CUDA-graph replay of the library (one persistent launch each)


def step_launches(n, groups, persistent):
    """Step-kernel launches of one lbm_step(n) / lbm_batch_step(n): one per step and launch
    group, or, stepping persistently, one per run of up to GRAPH_STEPS steps."""
    if persistent:
        return groups * (n // GRAPH_STEPS + (1 if n % GRAPH_STEPS else 0))
    return groups * n


def load_traffic(n_nodes, block_size, profile="sweep2_kernel_fp32.md", tile=None,
                 stepping=None):
    """DRAM bytes per step from a committed ncu summary of the step kernel, scaled to
    n_nodes, or None when the kernel source, its block size, (for a batch) its tiling or
    the way it steps ("persistent" or "per-step") has changed since that capture."""
    path = os.path.join(ROOT, "profiles", profile)
    vals = {}
    try:
        with open(path) as fh:
            for line in fh:
                for key in ("kernel_hash", "block_size", "tile", "stepping",
                            "dram_bytes_per_node"):
                    if line.strip().startswith(key + ":"):
                        vals[key] = line.split(":", 1)[1].strip().strip("`")
    except OSError:
        return None
    if vals.get("kernel_hash") != kernel_source_hash() or "dram_bytes_per_node" not in vals:
        return None
    if vals.get("block_size") != str(block_size):
        return None
    if tile is not None and vals.get("tile") != tile:
        return None
    if stepping is not None and vals.get("stepping") != stepping:
        return None
    return float(vals["dram_bytes_per_node"]) * n_nodes


def load_fp64_flops():
    """FP64 flops per lattice update of the FP64 step kernel from the committed ncu
    summary (dadd + dmul + 2 dfma), or None when the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", "sweep_kernel_fp64.md")
    vals = {}
    try:
        with open(path) as fh:
            for line in fh:
                for key in ("kernel_hash", "fp64_flops_per_lu"):
                    if line.strip().startswith(key + ":"):
                        vals[key] = line.split(":", 1)[1].strip().strip("`")
    except OSError:
        return None
    if vals.get("kernel_hash") != kernel_source_hash("fp64") or "fp64_flops_per_lu" not in vals:
        return None
    return float(vals["fp64_flops_per_lu"])


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    """The largest v over the ranks (a host number; a CUDA tensor under NCCL, a CPU one
    under gloo)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(steps=None, budget_s=25.0):
    """The FP64 oracle on a 1024 x 1024 window of the workload, on the host cores: as many
    steps as budget_s seconds allow by the first step's time (10 to 2000; later steps run
    about twice as fast, so the sample takes roughly half the budget)."""
    import numpy as np

    import oracle
    from oracle import thermo
    T = eos_T()
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    rho = ref_field(rl, rv)
    p = oracle.Params(nx=REF_WINDOW, ny=REF_WINDOW, a=A, b=B, R=R, T=T, sigma=SIGMA,
                      s=RATES, visc_mode=oracle.VISC_LINEAR, nu_l=NU_L, nu_v=NU_V,
                      rho_l=rl, rho_v=rv)
    f = oracle.equilibrium(rho)
    f = oracle.run(p, f, 1)  # warm-up
    if steps is None:
        t0 = time.perf_counter()
        f = oracle.run(p, f, 1)
        one = time.perf_counter() - t0
        steps = max(10, min(2000, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    f = oracle.run(p, f, steps)
    dt = time.perf_counter() - t0
    assert np.isfinite(f).all()
    mlups = REF_WINDOW * REF_WINDOW * steps / dt / 1e6
    return {"value": mlups, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d oracle steps on the same recipe at %dx%d with 4 droplets (%.1f s)" % (
                steps, REF_WINDOW, REF_WINDOW, dt)}, steps, dt


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from oracle import thermo
    import numpy as np
    T = eos_T()
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    rho = ref_field(rl, rv)
    p = oracle.Params(nx=REF_WINDOW, ny=REF_WINDOW, a=A, b=B, R=R, T=T, sigma=SIGMA,
                      s=RATES, visc_mode=oracle.VISC_LINEAR, nu_l=NU_L, nu_v=NU_V,
                      rho_l=rl, rho_v=rv)
    f = oracle.equilibrium(rho)
    f = oracle.run(p, f, args.warmup)
    # the K steps in one oracle call, as the CPU baseline times it (no per-step transfer
    # of the populations between Python and the C oracle)
    t0 = time.perf_counter()
    f = oracle.run(p, f, args.steps)
    dt = time.perf_counter() - t0
    assert np.isfinite(f).all()
    value = REF_WINDOW * REF_WINDOW * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config({"sample_grid": [REF_WINDOW, REF_WINDOW], "sample_droplets": 4}),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.threads(),
                             "kind": "oracle",
                             "sample": "%d oracle steps (one call) of the same recipe at "
                                       "%dx%d with 4 droplets" % (args.steps, REF_WINDOW,
                                                                  REF_WINDOW)},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


BATCH_SCREEN = 10000  # --batch-screen


def batch256_instances():
    """The batched-equilibria recipe with the instances that turn non-finite within
    BATCH_SCREEN steps (a screen, untimed) left out: (instances, fields, total nodes,
    screen record)."""
    from paper_1211_6932_gb300 import batched
    insts, fields, draws = batched.instances(256, seed=4)
    t0 = time.perf_counter()
    bad = batched.screen(insts, fields, steps=BATCH_SCREEN) if BATCH_SCREEN > 0 else []
    keep = [i for i in range(len(insts)) if i not in bad]
    rec = {"screen_steps": BATCH_SCREEN, "retired_unstable": bad,
           "retired_draws": [{k: draws[i][k] for k in ("nx", "ny", "a", "T_over_Tc", "sigma",
                                                        "visc_ratio", "kind")} for i in bad],
           "screen_s": time.perf_counter() - t0}
    insts = [insts[i] for i in keep]
    fields = [fields[i] for i in keep]
    return insts, fields, sum(i.nx * i.ny for i in insts), rec


def run_batch(args):
    """--workload batch256: every instance advances one step per launch."""
    import torch

    from paper_1211_6932_gb300 import Batch

    from paper_1211_6932_gb300.sharding import shard

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    insts, fields, n_total, screen = batch256_instances()
    # the instances are independent: each rank advances its own share, no collective on
    # the data path (total work fixed: strong scaling)
    own = shard([i.nx * i.ny for i in insts], world, rank)
    insts = [insts[i] for i in own]
    fields = [fields[i] for i in own]
    n_nodes = sum(i.nx * i.ny for i in insts)
    stream = torch.cuda.Stream(device=dev)
    b = Batch(insts, precision="fp32", stream=stream)
    for i, rho in enumerate(fields):
        b.init_fields(i, rho)
    nt, vec, rows, tuned_ms = b.autotune(steps=64)
    per_step = b.launches_per_step  # launch groups, or 1 stepping persistently
    for _ in range(args.warmup):
        b.step(1)
    b.step(64)
    b.diagnostics()
    K = args.steps
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    step_ms = 0.0
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    # the diagnostics pass: one moments launch per kind of strip present (full-width for
    # instances of at most two columns per thread of its 128-thread CTAs) and the reduction
    mom_nt = 128 if nt < 0 else nt
    stored_nx = [i.ny if b.is_transposed(k) else i.nx for k, i in enumerate(insts)]
    diag_launches = 1 + len({nx <= 2 * mom_nt for nx in stored_nx}) if vec == 2 else 2
    k = 0
    launches = 0
    while k < K:
        n = min(DIAG_EVERY, K - k)
        e0.record(stream)
        b.step(n)
        e1.record(stream)
        e1.synchronize()
        step_ms += e0.elapsed_time(e1)
        launches += step_launches(n, per_step, b.persistent)
        if n == DIAG_EVERY:
            b.diagnostics()
            launches += diag_launches
        k += n
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    nonfinite = sum(d["nonfinite"] for d in b.diagnostics())
    total_ms = max_over_ranks(t0.elapsed_time(t1), world)
    peak, peak_kind = load_peak()
    avg = step_ms / K
    achieved = BYTES_PER_LU * n_nodes / (avg * 1e-3) / 1e9
    traffic = (load_traffic(n_nodes, nt, "sweep2_kernel_batch256.md", "%d,%d,%d" % (nt, vec, rows),
                            "persistent" if b.persistent else "per-step")
               if nt > 0 else None)
    if rank == 0:
        line = {"metric": "MLUPS (D2Q9 MRT-pseudopotential step, 256-instance batch, FP32)",
                "value": n_total * K / (total_ms * 1e-3) / 1e6, "unit": "MLUPS",
                "n_gpus": world, "steps": K, "warmup": args.warmup,
                "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "batch256_64to512_fp32", "instances": 256,
                           "instances_timed": 256 - len(screen["retired_unstable"]),
                           "screen": screen, "nonfinite_nodes_after": nonfinite,
                           "nodes": n_total, "nodes_rank0": n_nodes,
                           "tile_threads": "per_instance" if nt < 0 else nt,
                           "launches_per_step": per_step, "tile_vec": vec,
                           "transposed_instances": sum(map(b.is_transposed, range(len(insts)))),
                           "tile_rows": rows, "autotuned_ms": tuned_ms,
                           "diag_every": DIAG_EVERY,
                           "l2": "state %.2f GB > 129 MB L2, no flush" % (72 * n_nodes / 1e9),
                           "parallelism": ("instances sharded over %d ranks" % world
                                           if world > 1 else "one GPU")},
                "gpu_launches": launches,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                             "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                             "traffic_scope": "per step (every launch of one step)",
                             "peak_source": peak_kind, "avg_step_ms": avg,
                             "persistent": b.persistent},
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    b.close()
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    from paper_1211_6932_gb300 import Eos, Lattice, maxwell

    world, rank, local = dist_setup()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    T = eos_T()
    eos = Eos(a=A, T=T, b=B, R=R)
    rl, rv = maxwell(eos)
    rho = field(rl, rv)
    stream = torch.cuda.Stream(device=dev)
    L = Lattice(NX, NY, eos, G=-1.0, sigma=SIGMA, s=RATES, nu_l=NU_L, nu_v=NU_V,
                precision=PREC, visc_mode="linear", stream=stream,
                tile_threads=args.tile_threads, tile_vec=args.tile_vec,
                tile_rows=args.tile_rows)
    L.init_fields(rho)
    n_nodes = NX * NY

    # warm-up (graph capture happens here)
    for _ in range(args.warmup):
        L.step(1)
    L.step(64)
    L.diagnostics()
    L.sync()

    K = args.steps
    chunks = []
    k = 0
    while k < K:
        n = min(DIAG_EVERY, K - k)
        chunks.append(n)
        k += n
    ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in chunks]
    ev_diag = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in chunks]
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    launches = 0
    diag_last = None
    t_all0.record(stream)
    persistent = L.persistent
    for i, n in enumerate(chunks):
        ev_step[i][0].record(stream)
        L.step(n)
        ev_step[i][1].record(stream)
        launches += step_launches(n, 1, persistent)
        if n == DIAG_EVERY:
            ev_diag[i][0].record(stream)
            diag_last = L.diagnostics()
            ev_diag[i][1].record(stream)
            launches += 2
    t_all1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    L.sync()
    total_ms = t_all0.elapsed_time(t_all1)
    step_ms = sum(a.elapsed_time(b) for a, b in ev_step)
    total_ms_max = max_over_ranks(total_ms, world)
    avg_launch_ms = step_ms / K
    value = world * n_nodes * K / (total_ms_max * 1e-3) / 1e6

    # End to end through the C ABI with host buffers: upload the initial fields from
    # pinned memory, 100 steps, read the density back, every cycle.  Host buffers are in
    # the storage precision (float32 for FP32).  The transfers are the asynchronous ones
    # (lbm_init_fields_async / lbm_moments_async): each cycle's upload and read-back run on
    # the handle's copy streams while neighbouring cycles step; the timed region ends when
    # the last read-back has landed (lbm_sync).
    e2e_steps = max(1, min(5, K // DIAG_EVERY))
    hdt = np.float32 if PREC == "fp32" else np.float64
    rho_h = torch.from_numpy(rho.astype(hdt)).pin_memory()
    out_h = torch.empty((NY, NX), dtype=torch.float32 if PREC == "fp32"
                        else torch.float64).pin_memory()
    rho_np, out_np = rho_h.numpy(), out_h.numpy()
    L.init_fields_async(rho_np)
    L.step(DIAG_EVERY)
    L.moments_async(out_np)
    L.sync()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        L.init_fields_async(rho_np)
        L.step(DIAG_EVERY)
        L.moments_async(out_np)
    L.sync()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = world * n_nodes * DIAG_EVERY * e2e_steps / e2e_s / 1e6

    peak, peak_kind = load_peak()
    bytes_lu = BYTES_PER_LU * (2 if PREC == "fp64" else 1)
    achieved = bytes_lu * n_nodes / (avg_launch_ms * 1e-3) / 1e9
    nt, vec, rows = L.tiling
    traffic = (load_traffic(n_nodes, nt, stepping="persistent" if persistent else "per-step")
               if vec == 2 and PREC == "fp32" else None)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if PREC == "fp32" else "f64",
            "data": "synthetic",
            "config": config({"tile_threads": nt, "tile_vec": vec, "tile_rows": rows}),
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_kind,
                         "kernel": (("sweep2_persist_kernel<%d>" if persistent
                                     else "sweep2_kernel<%d,STEP>") % nt if vec == 2
                                    else "sweep_kernel<%s,%d,STEP>"
                                    % ("float" if PREC == "fp32" else "double", nt)),
                         "persistent": persistent,
                         # per time step: stepping persistently, one launch runs up to
                         # GRAPH_STEPS steps (bytes and duration scale together)
                         "algorithmic_bytes_per_step": bytes_lu * n_nodes,
                         "avg_step_ms": avg_launch_ms,
                         "steps_per_launch": GRAPH_STEPS if persistent else 1},
            "e2e": {"value": e2e_value, "unit": "MLUPS",
                    "h2d_bytes_per_step": n_nodes * rho_h.element_size(),
                    "d2h_bytes_per_step": n_nodes * out_h.element_size(),
                    "lbm_steps_per_step": DIAG_EVERY},
            "clocks": clocks,
            "diagnostics": diag_last,
        }
        if PREC == "fp64":
            flops = load_fp64_flops()
            if flops is not None:
                tf = flops * n_nodes / (avg_launch_ms * 1e-3) / 1e12
                line["roofline_fp64"] = {"bound": "alu", "achieved": tf,
                                         "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                                         "frac": tf / FP64_NOMINAL_TFLOPS,
                                         "peak_source": "nominal FP64 rate",
                                         "fp64_flops_per_lu": flops}
        print("gpu part: %s" % json.dumps(line), file=sys.stderr, flush=True)
        if not args.no_other_workloads and world == 1 and NX == 4096:
            try:
                line["other_workloads"] = other_workloads(stream)
            except Exception as exc:  # reported, never hidden
                line["other_workloads"] = {"error": repr(exc)}
            print("other workloads: %s" % json.dumps(line["other_workloads"]), file=sys.stderr,
                  flush=True)
        if not args.no_other_workloads and world == 1 and NX == 4096:
            try:
                line["coexistence"] = coexistence_summary(stream)
            except Exception as exc:  # reported, never hidden
                line["coexistence"] = {"error": repr(exc)}
            try:
                line["interface"] = interface_summary(stream)
            except Exception as exc:  # reported, never hidden
                line["interface"] = {"error": repr(exc)}
            try:
                line["stability"] = stability_summary(stream)
            except Exception as exc:  # reported, never hidden
                line["stability"] = {"error": repr(exc)}
            try:
                line["calibration"] = calibration_summary(stream)
            except Exception as exc:  # reported, never hidden
                line["calibration"] = {"error": repr(exc)}
            try:
                line["dynamics"] = dynamics_summary(stream)
            except Exception as exc:  # reported, never hidden
                line["dynamics"] = {"error": repr(exc)}
        if not args.no_other_workloads and world == 1 and NX == 4096:
            try:
                line["batch_equilibrium"] = batch_equilibrium_summary(stream)
            except Exception as exc:  # reported, never hidden
                line["batch_equilibrium"] = {"error": repr(exc)}
            print("batch equilibrium: %s" % json.dumps(line["batch_equilibrium"]),
                  file=sys.stderr, flush=True)
        if not args.no_precision and world == 1 and NX == 4096:
            try:
                line["precision_error"] = precision_summary(stream)
            except Exception as exc:  # reported, never hidden
                line["precision_error"] = {"error": repr(exc)}
            print("precision: %s" % json.dumps(line["precision_error"]), file=sys.stderr,
                  flush=True)
        if not args.no_warm_start and world == 1 and NX == 4096:
            try:
                line["warm_start"] = warm_start_ab(stream)
            except Exception as exc:  # reported, never hidden
                line["warm_start"] = {"error": repr(exc)}
            print("warm start: %s" % json.dumps(line["warm_start"]), file=sys.stderr, flush=True)
        if not args.no_cpu_baseline:
            try:
                line["cpu_baseline"] = cpu_baseline()[0]
            except Exception as exc:  # reported, never hidden
                line["cpu_baseline"] = {"error": repr(exc)}
        print(json.dumps(line), flush=True)
    L.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def other_workloads(stream):
    """MLUPS of the other configurations, reported beside the headline (not roofline
    evidence: the 128^2 droplet is latency-bound, the ellipse and the splash fit in L2), of
    the FP64 parity mode on the 4096^2 field (144 B per lattice update) and of the
    256-instance batch (autotuned,
    640 graph-replayed steps).  Each: 3 warm-up steps and a 64-step graph
    capture, then `steps` steps timed with CUDA events on the lattice's stream."""
    import torch

    from paper_1211_6932_gb300 import Eos, Lattice, maxwell
    from paper_1211_6932_gb300 import workloads as wl
    out = []

    def timed(name, L, steps, n_nodes, dtype, bytes_per_lu, note, tune=False):
        if tune:  # the library's autotuner (untimed; state and step count restored)
            L.autotune(steps=64)
        L.step(3)
        L.step(64)
        L.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.step(steps)
        e1.record(stream)
        e1.synchronize()
        L.sync()
        ms = e0.elapsed_time(e1) / steps
        peak, kind = load_peak()
        rec = {"workload": name, "nodes": n_nodes, "dtype": dtype, "steps": steps,
               "ms_per_step": ms, "mlups": n_nodes / (ms * 1e-3) / 1e6,
               "hbm_frac": bytes_per_lu * n_nodes / (ms * 1e-3) / 1e9 / peak,
               "peak_source": kind, "note": note, "tiling": list(L.tiling)}
        flops = load_fp64_flops() if dtype == "f64" else None
        if flops is not None:
            tf = flops * n_nodes / (ms * 1e-3) / 1e12
            rec["fp64_tflops"] = tf
            rec["fp64_frac_of_nominal"] = tf / FP64_NOMINAL_TFLOPS
        out.append(rec)

    tau8 = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.25, 1.25)  # Sec. IV A, tau_nu = 0.8
    # 128^2 stationary droplet, FP64
    e = Eos(a=0.25, T=0.7 * wl.t_crit(0.25))
    rl, rv = maxwell(e)
    with Lattice(128, 128, e, sigma=0.114, s=tau8, precision="fp64", stream=stream) as L:
        L.init_fields(wl.droplet(128, 128, rl, rv, 30.0, 4.0))
        timed("droplet_128x128_fp64", L, 5000, 128 * 128, "f64", 144,
              "1.2 MB of state: latency-bound; autotuned tiling", tune=True)
    # 1024^2 oscillating ellipse, linear viscosity
    e = Eos(a=0.25, T=0.6 * wl.t_crit(0.25))
    rl, rv = maxwell(e)
    with Lattice(1024, 1024, e, sigma=0.114, s=RATES, nu_l=0.05, nu_v=0.5,
                 visc_mode="linear", precision="fp32", stream=stream) as L:
        L.init_fields(wl.ellipse(1024, 1024, rl, rv, 240, 160, 4.0, noise=1e-4, seed=2))
        timed("ellipse_1024x1024_fp32", L, 2000, 1024 * 1024, "f32", 72,
              "75 MB of state: L2-resident; autotuned tiling", tune=True)
    # 2048 x 512 splash with walls, step viscosity, Re = 200, ratio 15
    e = Eos(a=0.25, T=0.5 * wl.t_crit(0.25))
    rl, rv = maxwell(e)
    nu_l = 0.05 * 160 / 200
    with Lattice(2048, 512, e, sigma=0.114, s=(1.0, 0.8, 0.8, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0),
                 nu_l=nu_l, nu_v=15 * nu_l, visc_mode="step", bc="walls", precision="fp32",
                 stream=stream) as L:
        rho, ux, uy = wl.splash(2048, 512, rl, rv, 4.0, 32, 160, 0.05)
        L.init_fields(rho, ux, uy)
        timed("splash_2048x512_walls_fp32", L, 2000, 2048 * 512, "f32", 72,
              "75 MB of state: L2-resident; autotuned tiling", tune=True)
    # the 4096^2 field, FP32 storage with psi of Eq. 24 evaluated in FP64 (psi_fp64 option)
    e = Eos(a=A, T=eos_T(), b=B, R=R)
    rl, rv = maxwell(e)
    with Lattice(NX, NY, e, sigma=SIGMA, s=RATES, nu_l=NU_L, nu_v=NU_V, visc_mode="linear",
                 precision="fp32", psi_fp64=True, stream=stream) as L:
        L.init_fields(field(rl, rv))
        timed("droplets64_%dx%d_fp32_psi_fp64" % (NX, NY), L, 500, NX * NY, "f32", 72,
              "FP32 storage and arithmetic, psi in FP64")
    # the 4096^2 field in the FP64 parity mode
    e = Eos(a=A, T=eos_T(), b=B, R=R)
    rl, rv = maxwell(e)
    with Lattice(NX, NY, e, sigma=SIGMA, s=RATES, nu_l=NU_L, nu_v=NU_V, visc_mode="linear",
                 precision="fp64", stream=stream) as L:
        L.init_fields(field(rl, rv))
        timed("droplets64_%dx%d_fp64" % (NX, NY), L, 200, NX * NY, "f64", 144,
              "FP64 populations and arithmetic (the 1e-12 parity mode)")
    # the 256-instance batch (autotuned tiling), one GPU
    from paper_1211_6932_gb300 import Batch
    insts, fields, n_total, screen = batch256_instances()
    b = Batch(insts, precision="fp32", stream=stream)
    try:
        for i, rho in enumerate(fields):
            b.init_fields(i, rho)
        nt, vec, rows, _ = b.autotune(steps=64)
        b.step(3)
        b.step(64)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(640)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 640
        bad = sum(d["nonfinite"] for d in b.diagnostics())
        peak, kind = load_peak()
        out.append({"workload": "batch256_64to512_fp32", "nodes": n_total, "dtype": "f32",
                    "steps": 640, "ms_per_step": ms, "mlups": n_total / (ms * 1e-3) / 1e6,
                    "hbm_frac": 72 * n_total / (ms * 1e-3) / 1e9 / peak, "peak_source": kind,
                    "note": "%d of 256 ragged instances (the ones that stay finite over a "
                            "10^4-step screen), %.2f GB of state"
                            % (len(insts), 72 * n_total / 1e9),
                    "retired_unstable": screen["retired_unstable"],
                    "tiling": ["per_instance" if nt < 0 else nt, vec, rows],
                    "launches_per_step": b.launches_per_step, "nonfinite_nodes": bad})
    finally:
        b.close()
    return out


def coexistence_summary(stream):
    """Fig. 1 of the paper as one batch of flat films (a = 0.5; sigma 0 and 0.11; tau_nu
    0.6 and 0.8; T/Tc 0.49 .. 0.95; 40000 steps): lowest stable reduced temperature and
    largest deviation from the Maxwell densities per scheme."""
    from paper_1211_6932_gb300 import coexistence as cx
    t0 = time.perf_counter()
    pts = cx.sweep(a=0.5, steps=40000, stream=stream)
    secs = time.perf_counter() - t0
    out = {"films": len(pts), "seconds": secs, "schemes": []}
    for sig in (0.0, 0.11):
        for tau in (0.6, 0.8):
            ok = [p for p in pts if p.sigma == sig and p.tau_nu == tau and p.stable]
            out["schemes"].append({
                "sigma": sig, "tau_nu": tau, "lowest_stable_T_over_Tc": cx.lowest_stable(pts, sig, tau),
                "max_rel_dev_liquid": max(abs(p.rho_l / p.maxwell_l - 1) for p in ok) if ok else None,
                "max_rel_dev_vapour": max(abs(p.rho_v / p.maxwell_v - 1) for p in ok) if ok else None})
    return out


def interface_summary(stream):
    """Sec. IV B as one batch (films and 200^2 droplets for a = 1, 0.5, 0.25 at T/Tc 0.5 and
    0.55, 30000 steps): integral widths and the droplets' largest spurious velocity."""
    from paper_1211_6932_gb300 import interface as itf
    t0 = time.perf_counter()
    rows = itf.study(t_over_tc=(0.5, 0.55), steps=30000, stream=stream)
    return {"seconds": time.perf_counter() - t0,
            "rows": [{"a": r.a, "T_over_Tc": r.t_over_tc, "width": r.width, "max_u": r.max_u,
                      "density_ratio": r.density_ratio, "stable": r.stable} for r in rows]}


def stability_summary(stream):
    """Sec. IV C / Fig. 4 as batched multi-section on the 600 x 250 splash: for each
    viscosity ratio the bracket of the lowest liquid viscosity that stays finite and
    positive to t* = 3."""
    from paper_1211_6932_gb300 import stability as st
    t0 = time.perf_counter()
    br = st.lowest_stable_viscosity(stream=stream)
    out = {"seconds": time.perf_counter() - t0, "t_star": 3.0,
           "brackets": [{"ratio": b.ratio, "unstable_nu_l": b.unstable, "stable_nu_l": b.stable}
                        for b in br]}
    # the same search at the printed ratios under other readings of the paper's setup
    readings = {"finite_t6": {"t_star": 6.0}, "psi_real": {"criterion": "psi_real"},
                "umax_0.3": {"criterion": "umax"}, "sharp_velocity": {"velocity": "sharp"},
                "gap_0": {"gap": 0.0}, "gap_40": {"gap": 40.0}}
    out["readings"] = {}
    for name, kw in readings.items():
        rb = st.lowest_stable_viscosity(ratios=(1.0, 20.0, 50.0), stream=stream, **kw)
        out["readings"][name] = [{"ratio": b.ratio, "unstable_nu_l": b.unstable,
                                  "stable_nu_l": b.stable} for b in rb]
    out["printed"] = {"1": 0.075, "20": 0.009, "50": 0.0039}
    out["seconds_total"] = time.perf_counter() - t0
    return out


def calibration_summary(stream):
    """sigma of the improved forcing that makes a flat lattice film's vapour density the
    Maxwell value, for a = 0.25, 0.5, 1 at T/Tc 0.6 and 0.8 (batched films), next to the
    continuum calibration through Eq. 21."""
    from paper_1211_6932_gb300 import calibration as cb
    t0 = time.perf_counter()
    res = cb.sigma_lattice([(a, tr) for a in (0.25, 0.5, 1.0) for tr in (0.6, 0.8)],
                           stream=stream)
    rows = []
    for c in res:
        try:
            s21 = cb.sigma_eq21(c.a, c.t_over_tc)
        except Exception:
            s21 = None
        rows.append({"a": c.a, "T_over_Tc": c.t_over_tc, "sigma_lattice": c.sigma,
                     "bracket": [c.lo, c.hi], "sigma_eq21": s21})
    return {"seconds": time.perf_counter() - t0, "rows": rows}


def dynamics_summary(stream):
    """The paper's dynamic checks: Laplace law, the Sec. IV A oscillation against Eq. 32,
    the splash spread coefficient at Re 200 and 1000."""
    from paper_1211_6932_gb300 import dynamics as dy
    t0 = time.perf_counter()
    lf = dy.laplace_law(stream=stream)
    osc = dy.ellipse_period(stream=stream)
    c200 = dy.splash_spread(re=200.0, stream=stream).c
    c1000 = dy.splash_spread(re=1000.0, stream=stream).c
    return {"seconds": time.perf_counter() - t0,
            "laplace": {"gamma": lf.gamma, "intercept": lf.intercept, "r2": lf.r2},
            "oscillation": {"period": osc.period, "lamb": osc.lamb, "printed": 2600},
            "splash_C": {"re200": c200, "re1000": c1000, "printed": 1.3}}


def batch_equilibrium_summary(stream):
    """The batched-equilibria recipe run as specified: all 256 instances in one batch until
    each meets max |d rho| < tol per 100 steps (FP32: 1e-6, the float reading of the
    1e-9 tolerance; unstable instances are retired on the way), at most 60000 steps; and
    the 24 smallest stable instances in the FP64 mode at the stated 1e-9 (at most 150000
    steps), with their FP32 (1e-6) phase densities compared against the FP64 (1e-9)
    ones."""
    import numpy as np

    from paper_1211_6932_gb300 import batched
    insts, fields, draws = batched.instances(256, seed=4)
    t0 = time.perf_counter()
    e32 = batched.run_to_equilibrium(insts, fields, tol=1e-6, max_steps=60000, stream=stream)
    t32 = time.perf_counter() - t0
    st = e32.steps
    conv = st[st >= 0]
    films = [i for i in range(256) if draws[i]["kind"] == "film"]
    out = {"fp32": {"tol": 1e-6, "max_steps": 60000, "seconds": t32,
                    "converged": int(len(conv)), "unstable": e32.unstable,
                    "unconverged": len(e32.unconverged),
                    "unconverged_films": len([i for i in e32.unconverged if i in films]),
                    "steps_median": float(np.median(conv)) if len(conv) else None,
                    "steps_p90": float(np.percentile(conv, 90)) if len(conv) else None,
                    "steps_max": int(conv.max()) if len(conv) else None,
                    "node_steps": e32.node_steps,
                    "mlups_run": e32.node_steps / t32 / 1e6}}
    stable = [i for i in range(256) if i not in e32.unstable]
    sub = sorted(stable, key=lambda i: insts[i].nx * insts[i].ny)[:24]
    si, sf = [insts[i] for i in sub], [fields[i] for i in sub]
    t0 = time.perf_counter()
    e64 = batched.run_to_equilibrium(si, sf, tol=1e-9, max_steps=150000, precision="fp64",
                                     stream=stream, keep_fields=True)
    t64 = time.perf_counter() - t0
    e32s = batched.run_to_equilibrium(si, sf, tol=1e-6, max_steps=150000, stream=stream,
                                      keep_fields=True)
    dl, dv = [], []
    for k, i in enumerate(sub):
        if e64.rho[k] is None or e32s.rho[k] is None:
            continue
        rl, rv = insts[i].rho_l, insts[i].rho_v
        l64, v64 = batched.phase_densities(e64.rho[k], rl, rv)
        l32, v32 = batched.phase_densities(e32s.rho[k], rl, rv)
        dl.append(abs(l32 / l64 - 1))
        dv.append(abs(v32 / v64 - 1))
    out["fp64_subset"] = {"instances": sub, "tol": 1e-9, "seconds": t64,
                          "converged": int((e64.steps >= 0).sum()),
                          "steps": e64.steps.tolist(),
                          "fp32_1e-6_steps": e32s.steps.tolist(),
                          "max_rel_diff_liquid_fp32_vs_fp64": max(dl) if dl else None,
                          "max_rel_diff_vapour_fp32_vs_fp64": max(dv) if dv else None}
    return out


def precision_summary(stream):
    """Error of the FP32 path against the FP64 mode (oracle-matched per step) after the
    stated step counts: the 1024^2 ellipse (20000 steps), the 2048 x 512 splash (30000
    steps, density ratio > 500; step viscosity as in Sec. IV C, and tau linear in rho) and
    the 4096^2 field (2000 steps); per workload the
    maximum relative density error, the coexistence (bulk liquid / vapour mean) errors and
    the sensitivity floor of the flow (FP64 from the float-rounded start against FP64),
    at evenly spaced checkpoints."""
    from paper_1211_6932_gb300 import precision as pr
    t0 = time.perf_counter()
    out = {"bounds": {"max_rel_density": 1e-4, "coexistence": 1e-3}, "workloads": []}
    for name, steps, cps in (("ellipse_1024", 20000, 4), ("splash_2048", 30000, 6),
                             ("splash_2048_linear", 30000, 6), ("field_4096", 2000, 2)):
        r = pr.fp32_error(name, steps=steps, checkpoints=cps, floor=True, stream=stream)
        keep = ("step", "max_rel_density", "liquid_rel", "vapour_rel", "mass_rel",
                "fp64_floor")
        r["history"] = [{k: h.get(k) for k in keep} for h in r["history"]]
        out["workloads"].append(r)
    out["seconds"] = time.perf_counter() - t0
    return out


def warm_start_ab(stream):
    """Learned warm start against Eq. 31 on the 4096^2 field: the training set from the
    batched equilibria (256 draws, one film and two droplets each), the network trained on
    the GPU, then both initialisations relaxed for WARM_HORIZON steps with the phase
    densities recorded every 100 steps.  Steps-to-equilibrium: the first check after
    which the vapour and liquid phase densities stay within the tolerances of the plain
    run's final values (mean over its last 20 % of checks)."""
    import numpy as np

    from paper_1211_6932_gb300 import Lattice, workloads as wl
    from paper_1211_6932_gb300 import warmstart as ws
    t0 = time.perf_counter()
    draws = wl.warm_draws(256, seed=6)
    ds = ws.equilibria(draws, max_steps=60000, stream=stream)
    t_data = time.perf_counter() - t0
    sur = ws.Surrogate(seed=0, stream=stream)
    t1 = time.perf_counter()
    losses = sur.fit(ds, steps=4000, lr=3e-3)
    t_train = time.perf_counter() - t1
    eos = ws.eos_of(A, TR)
    plain = ws.plain_params(eos)
    warm = sur.predict(A, TR, SIGMA, NU_V / NU_L)
    members = len(sur.nets)
    sur.close()
    cs, rs = wl.droplet_layout(NX, NY, n_droplets(), 40.0, 200.0, seed=5, gap=4 * ws.W_PLAIN)
    drops = ws.drops_array(cs, rs)
    thr = ws.phase_thresholds(plain)
    # arms: Eq. 31 at rest (the paper's start), and the learned warm start (network
    # parameters, curvature law, force-balanced start); the two half-way arms separate
    # what the network and the balanced start each contribute
    arms = (("plain", plain, False, False), ("warm", warm, True, True),
            ("plain_balanced", plain, False, True), ("network_at_rest", warm, True, False))
    rel = {}
    with Lattice(NX, NY, eos, sigma=SIGMA, s=RATES, nu_l=NU_L, nu_v=NU_V, precision="fp32",
                 visc_mode="linear", stream=stream) as L:
        for name, prm, cur, bal in arms:
            rel[name] = ws.relax(L, drops, prm, cur, thr, 100, WARM_HORIZON, balanced=bal)
    rp, rw = rel["plain"], rel["warm"]
    ref_v, ref_l = ws.tail_mean(rp.vap), ws.tail_mean(rp.liq)
    tols = [(0.01, 0.002), (0.01, 0.001), (0.005, 0.001), (0.005, 0.0005), (0.02, 0.005)]
    settle = []
    for tv, tl in tols:
        row = {"tol_vapour": tv, "tol_liquid": tl}
        for name in rel:
            row[name] = ws.settling_step(rel[name], ref_v, ref_l, tv, tl)
        a, b = row["plain"], row["warm"]
        row["saved"] = (a - b) if a is not None and b is not None else None
        settle.append(row)
    # size of the start-up ringing of each arm: the largest relative departure of the
    # liquid and vapour phase densities from the plain run's final values over early
    # (steps 500-5000) and late (10000-30000) windows
    def ringing(r, lo, hi):
        m = (r.steps >= lo) & (r.steps <= hi)
        return {"liquid": float(np.max(np.abs(r.liq[m] / ref_l - 1.0))),
                "vapour": float(np.max(np.abs(r.vap[m] / ref_v - 1.0)))}
    ring = {name: {"early": ringing(r, 500, 5000), "late": ringing(r, 10000, 30000),
                   "start_vapour": float(r.vap[0] / ref_v - 1.0),
                   "start_liquid": float(r.liq[0] / ref_l - 1.0)}
            for name, r in rel.items()}
    return {
        "metric": "warm-start steps saved (4096^2, 64 droplets, phase densities within "
                  "1 % vapour / 0.2 % liquid)",
        "value": settle[0]["saved"], "unit": "steps",
        "settling": settle,
        "ringing": ring,
        "start_error": {"plain_vapour": rp.vap[0] / ref_v - 1, "warm_vapour": rw.vap[0] / ref_v - 1},
        "final": {"plain_vapour": ref_v, "plain_liquid": ref_l,
                  "warm_vapour": ws.tail_mean(rw.vap), "warm_liquid": ws.tail_mean(rw.liq),
                  "rel_diff_vapour": ws.tail_mean(rw.vap) / ref_v - 1,
                  "rel_diff_liquid": ws.tail_mean(rw.liq) / ref_l - 1},
        "horizon": WARM_HORIZON, "thresholds": list(thr),
        "params": {"plain": plain.__dict__, "warm": warm.__dict__},
        "network": {"members": members, "updates": int(len(losses)),
                    "loss_first": float(losses[0]),
                    "loss_last": float(losses[-1]), "train_s": t_train},
        "dataset": {"draws": len(draws), "rows": int(len(ds.x)), "dropped": len(ds.dropped),
                    "unconverged": [int(v) for v in (ds.steps < 0).sum(axis=0)],
                    "seconds": t_data},
    }


def network_gemms():
    """The warm-start network's training update against the tensor-core route: device time
    of cuBLAS bf16 products (torch.matmul) of the update's eight shapes, each replayed 100
    times from a CUDA graph (10 replays timed with CUDA events on the replay stream), and
    the library's fused update (4000 updates of one network on 256 rows).  One JSON line."""
    import numpy as np
    import torch

    from paper_1211_6932_gb300 import workloads as wl
    from paper_1211_6932_gb300.mlp import Mlp
    rows, ni, nh, no = 256, 4, 64, 5
    shapes = [("forward", rows, ni, nh), ("forward", rows, nh, nh), ("forward", rows, nh, no),
              ("weight gradient", no, rows, nh), ("input gradient", rows, no, nh),
              ("weight gradient", nh, rows, nh), ("input gradient", rows, nh, nh),
              ("weight gradient", nh, rows, ni)]
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream(device=dev)
    products = []
    for kind, m, k, n in shapes:
        a = torch.randn(m, k, device=dev, dtype=torch.bfloat16)
        b = torch.randn(k, n, device=dev, dtype=torch.bfloat16)
        c = torch.empty(m, n, device=dev, dtype=torch.bfloat16)
        with torch.cuda.stream(st):
            for _ in range(3):
                torch.matmul(a, b, out=c)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            for _ in range(100):
                torch.matmul(a, b, out=c)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            g.replay()
            e0.record()
            for _ in range(10):
                g.replay()
            e1.record()
        torch.cuda.synchronize()
        products.append({"product": "%s %dx%dx%d" % (kind, m, k, n),
                         "us": e0.elapsed_time(e1) * 1e3 / 1000})
    rng = np.random.default_rng(0)
    x, y = rng.uniform(size=(rows, ni)), rng.normal(size=(rows, no))
    net = Mlp(wl.mlp_init(0), max_rows=4096)
    try:
        net.fit_scaling(x, y)
        net.set_data(x, y)
        net.train(100, lr=1e-3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.train(4000, lr=1e-3)
        torch.cuda.synchronize()
        update_us = (time.perf_counter() - t0) / 4000 * 1e6
    finally:
        net.close()
    print(json.dumps({"metric": "warm-start network update against cuBLAS bf16 products",
                      "products": products,
                      "products_sum_us": sum(p["us"] for p in products),
                      "fused_update_us": update_us}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--tile-threads", type=int, default=0)
    ap.add_argument("--tile-vec", type=int, default=0)
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the MLUPS of the other workloads (droplet, ellipse, splash, "
                         "batch) and of the FP64 mode")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the FP32-against-FP64 error over the stated runs (1 GPU only)")
    ap.add_argument("--no-warm-start", action="store_true",
                    help="skip the learned warm-start comparison (4096^2, 1 GPU only)")
    ap.add_argument("--workload", default="field4096", choices=["field4096", "batch256"],
                    help="field4096 (default): the 4096^2 droplet field; batch256: the "
                         "256-instance batched-equilibria recipe")
    ap.add_argument("--batch-screen", type=int, default=10000,
                    help="steps of the untimed instability screen of the 256-instance "
                         "batch (0: none; for short profiling runs)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="fp32 (default; the headline) or fp64 (the parity mode)")
    ap.add_argument("--grid", type=int, default=4096,
                    help="square grid side (default 4096; smaller grids for profiling)")
    ap.add_argument("--network-gemms", action="store_true",
                    help="only time the warm-start network's update against cuBLAS bf16 "
                         "products of its shapes (one JSON line)")
    args = ap.parse_args()
    global NX, NY, PREC, BATCH_SCREEN
    NX = NY = args.grid
    PREC = args.precision
    BATCH_SCREEN = args.batch_screen
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.network_gemms:
        return network_gemms()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch256":
        return run_batch(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
