"""Benchmark: geodesic 3x3 dilation chains on one GB300 (or N replicas).

A bench step is one 1500-step, 8-connected geodesic dilation chain
(f <- min(delta_1(f), mask), Zlaus & Mongus Eq. 3-4) on a 1024x1024 uint8
marker/mask pair from the seeded synthetic generator, through the C ABI
entry point geo_dilate_chain. The metric is Gpixel-steps/s =
H * W * chain_steps / seconds / 1e9, summed over all ranks (replicas).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --only {batched,fwd_bwd,reconstruct_4096,operators,workload1}

--only runs one of the secondary measurements alone (for profiler captures).

--impl reference times the CPU oracle (the plain C loops of oracle/) on the
host cores instead, on a bounded number of chain steps per bench step.
Prints one JSON line (rank 0).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 1024
CHAIN_STEPS = 1500
CONN = 8
OPS_PER_PX_STEP = 5  # 8-connected masked step: 2 row + 2 column extremes + 1 mask clamp
WORKLOAD = "1024x1024 uint8 8-connected geodesic dilation chain, 1500 steps (synthetic workload 1)"
METRIC = "Gpixel-steps/s (1024² u8, 1500-step geodesic chain)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="geomorph", choices=["geomorph", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-secondary", action="store_true",
                   help="skip the batched and forward+backward comparisons")
    p.add_argument("--only", default=None, choices=["batched", "fwd_bwd", "reconstruct_4096", "operators",
                                                    "workload1"],
                   help="run one secondary measurement alone (for profiler captures) and print it")
    p.add_argument("--write-traffic-record", nargs=2, metavar=("NCU_CSV", "OUT_JSON"), default=None,
                   help="write the chain kernel's DRAM traffic record from the CSV of the ncu capture "
                        "(TRAFFIC_COMMAND) and exit")
    p.add_argument("--chain-steps", type=int, default=CHAIN_STEPS,
                   help="chain length of a bench step (default 1500; shorter only for small profiler captures, "
                        "and then named in the output's config)")
    return p.parse_args()


def dist_setup(n):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
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
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# the sources that define the timed chain kernel (rr_kernel for uint8) and its launch
CHAIN_KERNEL_SOURCES = ("geo_common.cuh", "geo_tile.cuh", "geo_rr.cuh", "geo_launch.cuh", "geo_tile_u8.cu",
                        "geo_api.cu")


def kernel_source_sha256():
    import hashlib
    h = hashlib.sha256()
    for name in CHAIN_KERNEL_SOURCES:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_1911_13074_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic():
    """DRAM bytes per launch of the chain kernel from the committed ncu record,
    or None when the kernel sources changed since the counters were taken."""
    try:
        with open(TRAFFIC_RECORD) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("source_sha256") != kernel_source_sha256():
        return None
    return rec.get("traffic_bytes_per_launch")


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "rr_kernel_u8_1024_chain1500_traffic.json")
TRAFFIC_COMMAND = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                   "--clock-control none --print-units base -k regex:rr_kernel -s 1 -c 1 --csv --log-file <csv> "
                   "python bench.py --steps 1 --warmup 1 --no-secondary --no-cpu-baseline")


def write_traffic_record(csv_path, out_path):
    """Turn the ncu CSV of TRAFFIC_COMMAND (one captured launch of the timed
    chain kernel) into the traffic record bench.py reads, stamped with the
    SHA-256 of the chain kernel's sources as they are when this runs (right
    after the capture, on the same checkout)."""
    import csv
    vals, name = {}, None
    with open(csv_path, newline="") as fh:
        rows = [r for r in csv.reader(fh) if r]
    head = next(i for i, r in enumerate(rows) if "Metric Name" in r)
    cols = rows[head]
    for r in rows[head + 1:]:
        if len(r) != len(cols):
            continue
        d = dict(zip(cols, r))
        name = d.get("Kernel Name", name)
        vals[d["Metric Name"]] = (float(d["Metric Value"].replace(",", "")), d.get("Metric Unit", ""))
    rd, wr = vals["dram__bytes_read.sum"], vals["dram__bytes_write.sum"]
    dur = vals["gpu__time_duration.sum"]
    for v in (rd, wr):
        if v[1] not in ("byte", "bytes", ""):
            raise ValueError(f"unexpected unit {v[1]} (the capture takes --print-units base)")
    rec = {"kernel": name, "workload": "1024x1024 u8 workload 1, 1500-step chain, one launch (the timed launch "
                                       "of the command)",
           "command": TRAFFIC_COMMAND, "passes": 1,
           "dram_bytes_read": rd[0], "dram_bytes_write": wr[0], "traffic_bytes_per_launch": rd[0] + wr[0],
           "gpu_time_ms_under_ncu": dur[0] / 1e6 if dur[1].startswith("n") else dur[0],
           "source_sha256": kernel_source_sha256(),
           "note": "written by bench.py --write-traffic-record from the capture's CSV; source_sha256 is computed "
                   "from the chain kernel's sources at that moment"}
    with open(out_path, "w") as fh:
        json.dump(rec, fh, indent=1)
    return rec


def max_over_ranks(values, world, device=None):
    """Per-rank timings -> their maximum over all ranks (the slowest rank
    sets the whole job's time). One all-reduce on the process group's
    backend: CUDA tensors under NCCL, CPU tensors under gloo."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    dev = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def whole_job_rate(world, units_per_rank_step, steps, seconds):
    """Units all ranks processed (weak scaling: each rank a full workload per
    step) per second, in billions."""
    return world * units_per_rank_step * steps / seconds / 1e9


def alu_peak_top_s(nsm, lanes_per_clk, mhz):
    """Peak exact min/max rate for uint8 pixels, in tera pixel-ops per second.

    The fastest exact primitives for uint8 values on sm_103a are the packed
    max / min of two u16 lanes (max.u16x2, max.f16x2), each lane deciding one
    pixel of two. lanes_per_clk is their measured rate per SM clock (the
    library's probe: 64, half the issue rate of 128).
    """
    return nsm * lanes_per_clk * 2 * mhz * 1e6 / 1e12


# Fewest instructions per pixel-step of the fastest exact min/max form of
# each element path: uint8, two pixels per packed instruction, 5 operations
# a masked step (2 row + 2 column extremes + the clamp) and 4 unmasked; float32
# (and float64 through its ranks), one pixel per instruction, a 3-extreme in
# one three-input max.f32: 3 instructions a masked step, 2 unmasked.
INSTR_PER_PX_STEP = {("u8", True): 2.5, ("u8", False): 2.0, ("f32", True): 3.0, ("f32", False): 2.0}


def peak_px_steps(nsm, rate, mhz, kind, masked):
    """Peak pixel-steps per second of an element path: SMs x measured
    min/max rate (lanes per SM clock) x clock / instructions per pixel-step."""
    return nsm * rate * mhz * 1e6 / INSTR_PER_PX_STEP[(kind, masked)]


def dtype_fractions(sec, nsm, u8_rate, f32_rate, mhz):
    """Roofline fractions of the secondary measurements, each against its
    element path's peak (peak_px_steps)."""
    out = {}
    w1 = sec.get("workload1_1024", {})
    for name, v in w1.items():
        if not isinstance(v, dict):
            continue
        parts = name.split("_")
        kind, masked = parts[1], parts[0] == "chain"
        if kind == "f64":
            steps = int(parts[-1][5:]) if masked else int(parts[-1][1:])
            if not masked or steps < 160:
                continue  # int64-key path (no probed rate); from 160 steps the rank path runs the float32 kernel
            kind = "f32"
        peak = peak_px_steps(nsm, u8_rate if kind == "u8" else f32_rate, mhz, kind, masked)
        out[name] = {"gpixel_steps_per_s": v["gpixel_steps_per_s"], "peak_gpixel_steps_per_s": peak / 1e9,
                     "frac": v["gpixel_steps_per_s"] * 1e9 / peak,
                     "path": "float32 kernel on ranks (rank transform included in the time)"
                     if parts[1] == "f64" else kind}
    rec = sec.get("reconstruct_4096", {})
    try:
        with open(os.path.join(ROOT, "tests", "golden", "workload2_sha256.json")) as fh:
            golden = json.load(fh)["cases"]
    except (OSError, ValueError):
        golden = {}
    for kind in ("u8", "f32"):
        for name, gname in (("opening_31x31", "open15"), ("hdome_minus20", "hdome20")):
            v, g = rec.get(f"{kind}_{name}"), golden.get(f"rec_{kind}_{gname}_conn8")
            if not v or not g:
                continue
            # the plain method's work: every pixel for every changing step plus the step that changes nothing
            px = 4096 * 4096 * (g["oracle_changing_steps"] + 1)
            achieved = px / (v["ms"] / 1e3)
            peak = peak_px_steps(nsm, u8_rate if kind == "u8" else f32_rate, mhz, kind, True)
            out[f"reconstruct_4096_{kind}_{name}"] = {
                "algorithmic_steps": g["oracle_changing_steps"] + 1, "gpixel_steps_per_s": achieved / 1e9,
                "peak_gpixel_steps_per_s": peak / 1e9, "frac": achieved / peak}
    fb = sec.get("fwd_bwd")
    if fb:
        peak = peak_px_steps(nsm, f32_rate, mhz, "f32", True)
        out["workload4_plain_forward_f32"] = {"gpixel_steps_per_s": fb["plain_forward_gpixel_steps_per_s"],
                                              "peak_gpixel_steps_per_s": peak / 1e9,
                                              "frac": fb["plain_forward_gpixel_steps_per_s"] * 1e9 / peak}
    return out


def probe_alu(gm):
    """Lane-ops per SM clock of the faster packed min/max form, and the clock
    the probe ran at."""
    best = (0.0, 0.0, "")
    for form in ("u16x2", "f16x2"):
        rate, mhz = gm.probe_minmax_rate(form)
        if rate > best[0]:
            best = (rate, mhz, form)
    return best


# --- the oracle on the host cores: one process per core (spawned, so it is
# safe after the process has used the GPU), each running the oracle as it
# stands on the same workload; throughput is the sum over the processes ---

_ORACLE_INPUT = {}


def _oracle_init():
    import oracle
    import synth
    w = synth.workload1_u8(H, W)
    _ORACLE_INPUT["f"], _ORACLE_INPUT["m"] = w["marker_dilate"], w["mask"]
    oracle.build()


def _oracle_task(steps):
    import oracle
    t0 = time.perf_counter()
    oracle.chain(_ORACLE_INPUT["f"], _ORACLE_INPUT["m"], steps, conn=CONN)
    return time.perf_counter() - t0


class OraclePool:
    """n processes that each run oracle chains of the 1024^2 u8 workload."""

    def __init__(self, n=None):
        import multiprocessing
        import oracle
        oracle.build()  # once, before the workers load it
        self.n = n or os.cpu_count() or 1
        self.pool = multiprocessing.get_context("spawn").Pool(self.n, initializer=_oracle_init)
        self.pool.map(_oracle_task, [1] * self.n)  # load and warm every worker

    def run(self, steps):
        """Every worker runs a chain of `steps`; returns the wall time."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_task, [steps] * self.n, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def host_cpu():
    """(logical cores, CPU model name) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as fh:
                for ln in fh:
                    if ln.lower().startswith("model name"):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return os.cpu_count() or 1, model or "unknown"


def _omp_task(job):
    """In a spawned process: the OpenMP build of the oracle (rows of each step
    split over `threads` threads) runs one chain of `steps` on the workload;
    returns the wall time. OMP_NUM_THREADS is set before the OpenMP runtime
    starts (it starts when the library is first loaded in this process)."""
    steps, threads = job
    os.environ["OMP_NUM_THREADS"] = str(threads)
    import oracle
    import synth
    w = synth.workload1_u8(H, W)
    oracle.chain_openmp(w["marker_dilate"], w["mask"], 1, conn=CONN)  # load the library, start the threads
    t0 = time.perf_counter()
    oracle.chain_openmp(w["marker_dilate"], w["mask"], steps, conn=CONN)
    return time.perf_counter() - t0


class OmpOracle:
    """One spawned process (safe after this process has used the GPU) running
    the OpenMP oracle on every host core."""

    def __init__(self, threads=None):
        import multiprocessing
        import oracle
        oracle.build_openmp()  # once, before the worker loads it
        self.threads = threads or os.cpu_count() or 1
        self.pool = multiprocessing.get_context("spawn").Pool(1)

    def run(self, steps):
        return self.pool.apply(_omp_task, ((steps, self.threads),))

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args, rank, world):
    """CPU oracle, timed on the host cores on a bounded sample of the
    workload: each bench step is sample_steps steps of the chain, run by the
    OpenMP build of the oracle (the rows of every step split over all host
    cores: one chain on all cores)."""
    if rank != 0:
        return
    sample_steps = 150  # a tenth of the 1500-step chain per bench step
    nproc, model = host_cpu()
    omp = OmpOracle(nproc)
    for _ in range(args.warmup):
        omp.run(sample_steps)
    dt = sum(omp.run(sample_steps) for _ in range(args.steps))
    omp.close()
    value = H * W * sample_steps * args.steps / dt / 1e9
    sample = (f"1024x1024 u8 8-connected dilation chain, {sample_steps} of the 1500 steps per bench step, "
              f"one chain with the rows of each step split over {nproc} OpenMP threads ({model})")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gpixel-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "chain_steps_timed_per_step": sample_steps,
                   "threads": nproc, "conn": CONN},
        "cpu_baseline": {"value": value, "unit": "Gpixel-steps/s", "cores": nproc, "kind": "oracle",
                         "sample": sample, "cpu_model": model},
        "e2e": {"value": value, "unit": "Gpixel-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline():
    """The oracle as it stands on bounded samples of the workload (about 8 s
    each): one chain with the rows of every step split over all host cores
    (OpenMP), the headline figure; one single-threaded chain per core
    (independent chains, throughput); and one core."""
    import oracle
    import synth
    nproc, model = host_cpu()
    w = synth.workload1_u8(H, W)
    f, m = w["marker_dilate"], w["mask"]
    oracle.build()
    t0 = time.perf_counter()
    oracle.chain(f, m, 5, conn=CONN)
    per_step = (time.perf_counter() - t0) / 5
    n = max(5, min(400, int(8.0 / max(per_step, 1e-6))))
    t0 = time.perf_counter()
    oracle.chain(f, m, n, conn=CONN)
    dt1 = time.perf_counter() - t0
    pool = OraclePool()
    dt = pool.run(n)
    pool.close()
    omp = OmpOracle(nproc)
    per_omp = omp.run(5) / 5
    n_omp = max(5, min(1500, int(8.0 / max(per_omp, 1e-6))))
    dt_omp = omp.run(n_omp)
    omp.close()
    return {"value": H * W * n_omp / dt_omp / 1e9, "unit": "Gpixel-steps/s", "cores": nproc, "kind": "oracle",
            "sample": f"1024x1024 u8 8-connected dilation chain, {n_omp} of the 1500 steps, one chain with the "
                      f"rows of each step split over {nproc} OpenMP threads, {dt_omp:.1f} s",
            "cpu_model": model, "nproc": nproc,
            "independent_chains": {"value": pool.n * H * W * n / dt / 1e9, "cores": pool.n,
                                   "sample": f"{n} steps in each of {pool.n} single-threaded processes, "
                                             f"{dt:.1f} s"},
            "single_core": {"value": H * W * n / dt1 / 1e9, "cores": 1, "seconds": round(dt1, 2)}}


def _time(fn, reps, warmup=1):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def _graph_of(fn):
    """fn captured once in a CUDA graph (on a side stream, as torch requires)."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    return g


def part_batched(dev):
    """Workload 3 (512 items) in one launch vs 512 single-item calls: each
    form first with the planners' cost-model plans, then after autotuning the
    items (shape variant and K per item, kept per size class); the batched
    launch is captured once in a CUDA graph and the graph is replayed."""
    import torch
    import paper_1911_13074_gb300 as gm
    import synth
    w3 = synth.workload3()
    items = []
    for it in w3:
        items.append({"op": it["op"], "marker": torch.from_numpy(it["marker"]).to(dev),
                      "mask": torch.from_numpy(it["mask"]).to(dev),
                      "steps": 0 if it["steps"] < 0 else it["steps"], "conn": it["conn"]})
    chain_px_steps = sum(int(it["marker"].numel()) * it["steps"] for it in items if it["op"] in (0, 1))

    def measure():
        batch = gm.Batch(items).prepare()
        graph = _graph_of(batch.launch)
        t_b = _time(graph.replay, 3)
        batch.check()  # every item's status and the device status word

        def plain():
            for it, out in zip(items, batch.outs):
                op = it["op"]
                if op in (0, 1):
                    (gm.dilate_chain if op == 0 else gm.erode_chain)(it["marker"], it["mask"], it["steps"],
                                                                    conn=it["conn"], out=out, check=False)
                else:
                    gm.reconstruct(it["marker"], it["mask"], conn=it["conn"],
                                   op="dilate" if op == 2 else "erode", out=out, check=False)
        t_p = _time(plain, 3)
        del graph, batch
        return t_b, t_p

    t_batch_cm, t_plain_cm = measure()
    # autotuning: the shape and K of every item's single-image calls, then
    # the batch planner's pass-length policy on the batch itself
    t0 = time.perf_counter()
    gm.autotune(items)
    gm.Batch(items).autotune()
    tune_s = time.perf_counter() - t0
    t_batch, t_plain = measure()
    res = {"batched": {
        "workload": "512 items, H,W log-uniform [64,2048] (W not a multiple of 32), half u8 half f32, "
                    "steps U{8..1500}, 25% to stability, op and conn drawn per item (synthetic workload 3)",
        "graph": True, "autotuned": True, "autotune_seconds": tune_s,
        "ms_batched": t_batch * 1e3, "ms_plain_512_calls": t_plain * 1e3,
        "speed_ratio_vs_plain": t_plain / t_batch,
        "chain_items_gpixel_steps_per_s": chain_px_steps / t_batch / 1e9,
        "cost_model_plans": {"ms_batched": t_batch_cm * 1e3, "ms_plain_512_calls": t_plain_cm * 1e3,
                             "speed_ratio_vs_plain": t_plain_cm / t_batch_cm},
        "all_items_ok": True, "gpu_launches_batched": 2, "gpu_launches_plain": len(items)}}
    del items, w3
    torch.cuda.empty_cache()
    return res


def part_fwd_bwd(dev):
    """Workload 4 (32 x 512^2 f32, 256 steps) forward + backward vs the plain forward."""
    import torch
    import paper_1911_13074_gb300 as gm
    import synth
    res = {}
    w4 = synth.workload4()
    mk, ms, g = (torch.from_numpy(w4[k]).to(dev) for k in ("marker", "mask", "grad_out"))
    steps = 256
    fb = {}
    for C in (16, 32, 64):
        def fwd_bwd(C=C):
            out, ws = gm.chain_fwd_ckpt(mk, ms, steps, conn=8, ckpt_interval=C, check=False)
            gm.chain_backward(ms, g, ws, steps, conn=8, ckpt_interval=C, check=False)
        fb[C] = _time(fwd_bwd, 3)
    out1 = torch.empty_like(mk)

    def plain_fwd():
        for b in range(mk.shape[0]):
            gm.dilate_chain(mk[b], ms[b], steps, conn=8, out=out1[b], check=False)
    t_pf = _time(plain_fwd, 3)
    px = mk.numel() * steps
    res["fwd_bwd"] = {
        "workload": "32 x 512x512 float32, 8-connected 256-step dilation chain (synthetic workload 4)",
        "ms_plain_forward_32_calls": t_pf * 1e3,
        "plain_forward_gpixel_steps_per_s": px / t_pf / 1e9,
        "ms_fwd_bwd": {str(C): t * 1e3 for C, t in fb.items()},
        "speed_ratio_vs_plain_forward": {str(C): t_pf / t for C, t in fb.items()},
    }
    del mk, ms, g, w4
    torch.cuda.empty_cache()
    return res


def part_reconstruct_4096(dev):
    """Workload 2 (4096^2 blob masks): dilation by reconstruction to stability, both markers."""
    import torch
    import paper_1911_13074_gb300 as gm
    import synth
    w2 = synth.workload2()
    rec = {}
    for kind in ("u8", "f32"):
        mask = torch.from_numpy(w2["mask_u8" if kind == "u8" else "mask_f32"]).to(dev)
        markers = {"opening_31x31": gm.window_erode(mask, 15),
                   "hdome_minus20": torch.from_numpy(w2["hdome_marker_" + kind]).to(dev)}
        for name, marker in markers.items():
            out = torch.empty_like(marker)
            steps_box = {}

            def run():
                _, st = gm.reconstruct(marker, mask, conn=8, out=out, return_steps=True, check=False)
                steps_box["s"] = st
            t = _time(run, 3)
            n = int(steps_box["s"].item())
            rec[f"{kind}_{name}"] = {"ms": t * 1e3, "steps_applied": n,
                                     "gpixel_steps_per_s": mask.numel() * n / t / 1e9}
    res = {"reconstruct_4096": {
        "workload": "4096x4096 blob masks (synthetic workload 2), 8-connected dilation by reconstruction to "
                    "stability; steps_applied counts whole passes up to the first unchanged pass",
        **rec}}
    del w2
    torch.cuda.empty_cache()
    return res


def part_operators(dev):
    """The geodesic operators of the paper's Table 5 on the 1024^2 u8 workload-1 image."""
    import torch
    import paper_1911_13074_gb300 as gm
    import synth
    res = {}
    g = torch.from_numpy(synth.workload1_u8()["mask"]).to(dev)
    ops = {"hmax_h20": lambda: gm.hmax(g, 20, check=False), "dome_h20": lambda: gm.dome(g, 20, check=False),
           "hfill": lambda: gm.hfill(g, check=False), "raobj": lambda: gm.raobj(g, check=False),
           "open_rec_s15": lambda: gm.open_rec(g, 15, check=False), "qdt": lambda: gm.qdt(g, check=False),
           "pattern_spectrum_0_11": lambda: gm.granulometry(g, 11, check=False),
           "asf_11": lambda: gm.asf(g, 11, check=False)}
    res["operators_1024_u8"] = {"workload": "1024x1024 u8 workload-1 image, 8-connected",
                                **{k: {"ms": _time(fn, 3) * 1e3} for k, fn in ops.items()}}
    return res


def part_workload1(dev):
    """Every workload-1 case at 1024^2: chains of u8 and f64, both operations
    and connectivities, 100 / 500 / 1500 steps, and the windows s = 13, 91."""
    import torch
    import paper_1911_13074_gb300 as gm
    import synth
    res = {}
    for kind, w in (("u8", synth.workload1_u8()), ("f64", synth.workload1_f64())):
        mask = torch.from_numpy(w["mask"]).to(dev)
        out = torch.empty_like(mask)
        for op in ("dilate", "erode"):
            mk = torch.from_numpy(w["marker_" + op]).to(dev)
            fn = gm.dilate_chain if op == "dilate" else gm.erode_chain
            for conn in (4, 8):
                for n in (100, 500, 1500):
                    t = _time(lambda: fn(mk, mask, n, conn=conn, out=out, check=False), 2)
                    res[f"chain_{kind}_{op}_conn{conn}_steps{n}"] = {
                        "ms": t * 1e3, "gpixel_steps_per_s": mask.numel() * n / t / 1e9}
            win = gm.window_dilate if op == "dilate" else gm.window_erode
            for s in (13, 91):
                t = _time(lambda: win(mask, s, out=out, check=False), 2)
                res[f"window_{kind}_{op}_s{s}"] = {"ms": t * 1e3,
                                                   "gpixel_steps_per_s": mask.numel() * s / t / 1e9}
    return {"workload1_1024": {"workload": "1024x1024 synthetic workload 1 (u8 and f64), every chain and window "
                                           "case; L2 not flushed between repetitions", **res}}


# batched last: its autotuning fills the library's tune table (per size
# class), which the other parts would otherwise pick up
PARTS = {"fwd_bwd": part_fwd_bwd, "reconstruct_4096": part_reconstruct_4096, "operators": part_operators,
         "workload1": part_workload1, "batched": part_batched}


def secondary(dev):
    """The batched and forward+backward forms against the plain path, and the
    other workloads, on the same GPU. The timed calls are the asynchronous
    (unchecked) form; the device status word is read after each part."""
    import paper_1911_13074_gb300 as gm
    res = {}
    for name, fn in PARTS.items():
        res.update(fn(dev))
        st = gm.device_status()
        if st != 0:
            raise RuntimeError(f"device status {st} after the {name} measurements")
    return res


def main():
    args = parse()
    if args.write_traffic_record:
        print(json.dumps(write_traffic_record(*args.write_traffic_record)), flush=True)
        return
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    import numpy as np
    import torch
    import paper_1911_13074_gb300 as gm
    import synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if args.only:
        if rank == 0:
            print(json.dumps({"part": args.only, **PARTS[args.only](dev)}), flush=True)
        return
    w = synth.workload1_u8(H, W)
    marker_h = torch.from_numpy(w["marker_dilate"]).pin_memory()
    mask_h = torch.from_numpy(w["mask"]).pin_memory()
    marker = marker_h.to(dev)
    mask = mask_h.to(dev)
    out = torch.empty_like(marker)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    alu_rate, alu_mhz, alu_form = probe_alu(gm)  # roofline denominator, before the warm-up
    mix_rate, _ = gm.probe_minmax_rate("mix")  # the best two-pipe mix, the second denominator
    f32_rate, _ = gm.probe_minmax_rate("f32x3")  # the float32 paths' denominators
    for _ in range(args.warmup):
        gm.dilate_chain(marker, mask, args.chain_steps, conn=CONN, out=out, check=False)
    torch.cuda.synchronize(dev)
    if gm.device_status() != 0:
        raise RuntimeError("device status error during warm-up")

    # device-timed region: inputs resident, L2 flushed between timed chains
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)  # let nvidia-smi start sampling before the timed region
    barrier()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        gm.dilate_chain(marker, mask, args.chain_steps, conn=CONN, out=out, check=False)
        ev[i][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    per = [a.elapsed_time(b) for a, b in ev]  # ms
    t_dev = sum(per) / 1e3
    status = gm.device_status()
    if status != 0:
        raise RuntimeError(f"device status {status}")

    # end to end through the public API with host buffers, as a user calls it:
    # the checked call (it synchronises and reads the device status word)
    out_h = torch.empty_like(marker_h).pin_memory()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        mk = marker_h.to(dev, non_blocking=True)
        ms = mask_h.to(dev, non_blocking=True)
        gm.dilate_chain(mk, ms, args.chain_steps, conn=CONN, out=out)
        out_h.copy_(out, non_blocking=True)
    e1.record(stream)
    barrier()
    t_e2e = e0.elapsed_time(e1) / 1e3

    t_dev, t_e2e = max_over_ranks([t_dev, t_e2e], world, dev)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    px_steps = H * W * args.chain_steps
    value = whole_job_rate(world, px_steps, args.steps, t_dev)
    e2e_value = whole_job_rate(world, px_steps, args.steps, t_e2e)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0
    peak = alu_peak_top_s(nsm, alu_rate, sm_max)
    issue_peak = alu_peak_top_s(nsm, 128, sm_max)
    per_launch_s = statistics.mean(per) / 1e3
    achieved = px_steps * OPS_PER_PX_STEP / per_launch_s / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "Gpixel-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.chain_steps == CHAIN_STEPS else
                   WORKLOAD.replace(f"{CHAIN_STEPS} steps", f"{args.chain_steps} steps (shortened)"),
                   "H": H, "W": W, "chain_steps": args.chain_steps, "conn": CONN,
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "flushed between timed chains (256 MiB write, outside the events)"},
        "fps": args.steps / t_dev,
        "wall_s_timed_region": t_wall,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "Gpixel-steps/s", "h2d_bytes_per_step": 2 * H * W,
                "d2h_bytes_per_step": H * W},
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tpixel-op/s",
                     "frac": achieved / peak, "traffic": measured_traffic(),
                     "traffic_unit": "bytes per launch (dram read + write, ncu)",
                     "peak_basis": f"{nsm} SMs x {alu_rate:.1f} lane-ops/clk (max.{alu_form}, measured by "
                                   f"geo_probe_minmax_rate at {alu_mhz:.0f} MHz) x 2 px x {sm_max:.0f} MHz",
                     "ops_per_pixel_step": OPS_PER_PX_STEP,
                     "mix_peak": alu_peak_top_s(nsm, mix_rate, sm_max),
                     "frac_of_mix_peak": achieved / alu_peak_top_s(nsm, mix_rate, sm_max),
                     "mix_basis": f"{mix_rate:.1f} maxima per SM clock for max.u16x2 mixed 2:1 with an exact "
                                  f"FMA-pipe max (geo_probe_minmax_rate form 3)",
                     "issue_rate_peak": issue_peak, "frac_of_issue_rate_peak": achieved / issue_peak},
    }
    if not args.no_secondary and world == 1:
        sec = secondary(dev)
        line.update(sec)
        line["fractions"] = {
            "basis": f"per element path: {nsm} SMs x measured rate (u8 packed {alu_rate:.1f}, f32 three-input "
                     f"{f32_rate:.1f} lane-ops per SM clock) x {sm_max:.0f} MHz / instructions per pixel-step "
                     f"(u8 2.5 masked, 2 unmasked; f32 3 masked, 2 unmasked)",
            **dtype_fractions(sec, nsm, alu_rate, f32_rate, sm_max)}
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
