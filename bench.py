"""Benchmark of the generalized FrequencyHough search on GB300.

One step = the whole path on one synthetic strain series: peakmap (cuFFT + equaliser + peak
test + compaction), then the Hough maps of every analysis sub-band (differential accumulation,
running sum, store) with the per-band candidates, all through the library's C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gfh|reference] [--workload NAME]

Metric: Hough updates per second, one update = one peak drawn on one k row (sum over maps of
peaks in the map's band x k rows).  Prints one JSON line on rank 0.  Under torchrun each rank
searches its own series (independent data segments, seed + rank): weak scaling, no collective on
the data path.  `--impl reference` times the CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import pathlib
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = pathlib.Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_1810_09784_gb300 import ranks, workloads  # noqa: E402

PEAKS = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
HBM_PEAK = PEAKS.get("hbm_gbs", 6800.0)
HBM_PEAK_SRC = "measured" if "hbm_gbs" in PEAKS else "fallback"
SM_MAX_MHZ = PEAKS.get("sm_max_mhz", 2070.0)
# Shared-memory atomic peak: measured on this GPU by the library's probe kernel (conflict-free
# 32-bit atomicAdd, every SM busy) before the timed steps; MEASURED_PEAKS has no such entry.
_ATOMIC_PROBE = {}


def atomic_peak(ctx, stream):
    """(peak G atomics/s, probe record): the conflict-free rate measured once per process."""
    if "rec" not in _ATOMIC_PROBE:
        _ATOMIC_PROBE["rec"] = measure_smem_atomics(ctx, stream)
    rec = _ATOMIC_PROBE["rec"]
    return rec["conflict_free"]["gatomic_s"], rec


def atomic_roofline(ctx, stream, achieved):
    peak, rec = atomic_peak(ctx, stream)
    return {"bound": "smem_atomic", "kernel": "k_hough", "achieved": achieved, "peak": peak,
            "unit": "Gatomic/s", "frac": achieved / peak,
            "peak_source": (f"measured: conflict-free shared atomicAdd over all {rec['sms']} SMs "
                            f"(library probe, CUDA events), "
                            f"{rec['conflict_free']['atomics_per_clk_per_sm']:.2f}/clk/SM at "
                            f"{rec['clocks'].get('sm_mhz')} MHz"),
            "probe": rec,
            "algorithmic": "2 shared atomics per update (differential +1/-1)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gfh", choices=["gfh", "reference"])
    ap.add_argument("--workload", default="plain_paper",
                    choices=["plain_paper", "plain_small", "batched_n", "paper_grids", "uneven",
                             "proposer", "followup", "splice", "train"])
    ap.add_argument("--no-graph", action="store_true",
                    help="time direct calls only (default: the step is also replayed as a CUDA graph)")
    ap.add_argument("--tile", default=None, help="rows,cols,threads of the Hough tiles")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: leave out the batched_n, uneven and proposer sub-objects")
    ap.add_argument("--sequential", action="store_true",
                    help="also time one plan per map (always on for batched_n)")
    ap.add_argument("--eval-maps", type=int, default=51 * 196,
                    help="proposer: held-out maps for the recall measurement (multiple of 51)")
    ap.add_argument("--maps", type=int, default=0,
                    help="profiling aid: keep only this many sub-band maps, spread over the band")
    ap.add_argument("--only-n", type=float, default=None,
                    help="profiling aid: keep only the maps of this braking index")
    ap.add_argument("--batch", type=int, default=256,
                    help="train: images per AdamW step (smaller batches are a profiling aid)")
    return ap.parse_args()


def dist_env():
    return ranks.rank_env()


def workload(name, rank):
    fn = getattr(workloads, name)
    base = {"plain_paper": 2, "plain_small": 1, "batched_n": 1, "paper_grids": 1}[name]
    return fn(seed=ranks.rank_seed(base, rank))


def describe(name, spec, grids):
    if name == "plain_paper":
        return (f"plain_paper: white noise + 20 power-law injections, fs {spec.fs:g} Hz, "
                f"{spec.t_obs:g} s, T_FFT {spec.t_fft:g} s ({spec.n_fft} FFTs), 50-2000 Hz in "
                f"{len(grids)} sub-bands (100 Hz + 50 Hz peakmap extension), n = 5, "
                f"{grids[0]['n_k']} k rows, top candidate per 1 Hz")
    if name == "paper_grids":
        ns = sorted({g["n"] for g in grids})
        return (f"paper_grids: the plain_small peakmap (fs {spec.fs:g} Hz, {spec.t_obs:g} s, T_FFT "
                f"{spec.t_fft:g} s, 100-400 Hz) on the paper's grids: {len(ns)} braking indices of "
                f"Eq. dn_powlaws in [2.5, 7] and, per index, the Eq. dkeqn k grid for |fdot| "
                f"1e-4..1e-2 Hz/s as {len(grids)} uniform segments (<= 512 rows), all in one launch")
    if name == "batched_n":
        return (f"batched_n: the plain_small peakmap (fs {spec.fs:g} Hz, {spec.t_obs:g} s, T_FFT "
                f"{spec.t_fft:g} s, 100-400 Hz) searched at {len(grids)} braking indices n = 2.0..7.0 "
                f"(step 0.1) with 4000 -> 1000 k rows, one map per n, all in one launch")
    return (f"plain_small: fs {spec.fs:g} Hz, {spec.t_obs:g} s, T_FFT {spec.t_fft:g} s "
            f"({spec.n_fft} FFTs), 100-400 Hz, n = 5, {grids[0]['n_k']} k rows")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        rows = [l.split(", ") for l in pathlib.Path(self.f.name).read_text().splitlines() if l.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()) if rows else None,
                "samples": len(rows), "reasons": reasons}


def measure_smem_atomics(ctx, stream, reps=3, iters=16384, threads=1024):
    """Shared-memory atomicAdd throughput of this GPU (gfh_probe_smem_atomics), every mode timed
    with CUDA events on the library's stream, best of `reps`; the SM count is read from the device
    and the SM clocks sampled while the probe runs."""
    import torch
    sms = ctx.sms()
    blocks = 2 * sms                                   # 2048 threads per SM
    cycles = torch.zeros(blocks, dtype=torch.int64, device="cuda")
    sink = torch.zeros(blocks, dtype=torch.int32, device="cuda")
    out = {"sms": sms, "blocks": blocks, "threads": threads, "iters_per_thread": iters}
    sampler = ClockSampler(torch.cuda.current_device())
    with sampler, torch.cuda.stream(stream):
        for mode, name in ((0, "conflict_free"), (1, "same_address"), (2, "random")):
            best = None
            for r in range(reps + 1):
                sink.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.probe_smem_atomics(mode, blocks, threads, iters, cycles, sink)
                b.record(stream)
                b.synchronize()
                if not bool((sink == threads * iters).all()):
                    raise RuntimeError("shared-atomic probe lost updates")
                ms = a.elapsed_time(b)
                if r > 0 and (best is None or ms < best[0]):
                    best = (ms, float(cycles.max().item()))
            n = float(blocks) * threads * iters
            out[name] = {"gatomic_s": n / (best[0] * 1e-3) / 1e9,
                         "atomics_per_clk_per_sm": n / sms / best[1]}
    out["clocks"] = sampler.summary()
    return out


def profile_record(kernel):
    """The committed ncu record of `kernel` (profiles/traffic.json), or None when the kernel's
    source changed since the counters were taken."""
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    rec = json.loads(p.read_text()).get(kernel)
    if not rec:
        return None
    src = (ROOT / rec["source"]).read_bytes()
    return rec if hashlib.sha256(src).hexdigest() == rec["sha256"] else None


def traffic_for(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the kernel's
    source changed since the counters were taken."""
    rec = profile_record(kernel)
    return rec["bytes_per_launch"] if rec else None


def issue_roofline(updates_per_s, sms, sm_mhz):
    """k_hough against the SMs' instruction issue: warp instructions per update from the committed
    ncu record (all of the kernel's instructions) times the measured update rate, against 4 warp
    instructions per clock per SM at the SM clock sampled under load; None without a record."""
    rec = profile_record("k_hough")
    if not rec or "warp_inst_per_update" not in rec:
        return None
    achieved = updates_per_s * rec["warp_inst_per_update"] / 1e9
    peak = sms * 4 * sm_mhz * 1e6 / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "Gwarp-inst/s", "frac": achieved / peak,
            "warp_inst_per_update": rec["warp_inst_per_update"],
            "peak_source": f"{sms} SMs x 4 schedulers x {sm_mhz:.0f} MHz (sampled under load)"}




# ---------------------------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------------------------

def host_cpu():
    """(usable cores, CPU model) of this host."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return cores, model


_OW = {}


def _oracle_attach(names):
    """Worker start-up: attach the shared arrays (series, peak list) by name; one numpy thread."""
    from multiprocessing import shared_memory
    os.environ["OMP_NUM_THREADS"] = "1"
    for key, (name, dtype, n) in names.items():
        shm = shared_memory.SharedMemory(name=name)
        _OW[key + "_shm"] = shm
        _OW[key] = np.ndarray((n,), dtype=np.dtype(dtype), buffer=shm.buf)


def _oracle_peak_chunk(task):
    """Peaks of frames [i0, i1) of the shared series: the oracle's peakmap of that slice (frames
    are independent, so the union over slices is the peakmap of the whole series)."""
    from oracle import gfh_oracle as O
    i0, i1, fs, t_fft, lo, hi = task
    N = int(round(fs * t_fft))
    hop = N // 2
    fi, bj = O.peakmap(_OW["x"][i0 * hop:(i1 - 1) * hop + N], fs, t_fft, lo, hi)
    return fi.astype(np.int64) + i0, bj.astype(np.int64)


def _oracle_rows(task):
    """The oracle's k rows `rows` of one map on the shared peak list (each row on its own)."""
    from oracle import gfh_oracle as O
    fields, rows = task
    og = O.make_grid(O.Grid(**{k: v for k, v in fields.items() if k != "list"}))
    t0 = time.perf_counter()
    out = [O.hough_row(og, _OW["fi"], _OW["bj"], int(r)) for r in rows]
    return time.perf_counter() - t0, out


class OraclePool:
    """Spawned worker processes (spawn: safe after CUDA use) running the unmodified oracle on every
    host core: the peakmap split by frames, Hough rows split by rows; inputs in shared memory."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or host_cpu()[0]
        self.mp = mp.get_context("spawn")
        self.pool = None
        self.shms = []

    def _share(self, arrays):
        from multiprocessing import shared_memory
        names = {}
        for key, a in arrays.items():
            a = np.ascontiguousarray(a)
            shm = shared_memory.SharedMemory(create=True, size=max(1, a.nbytes))
            np.ndarray(a.shape, a.dtype, buffer=shm.buf)[...] = a
            self.shms.append(shm)
            names[key] = (shm.name, a.dtype.str, a.size)
        return names

    def start(self, arrays):
        self.close_pool()
        self.pool = self.mp.Pool(self.cores, initializer=_oracle_attach, initargs=(self._share(arrays),))
        return self

    def peakmap(self, x, fs, t_fft, lo, hi):
        """(fft_idx, bin) sorted by (bin, FFT), identical to O.peakmap(x, ...)."""
        self.start({"x": np.asarray(x, np.float32)})
        N = int(round(fs * t_fft))
        n_frames = (x.size - N) // (N // 2) + 1
        step = max(1, -(-n_frames // (4 * self.cores)))
        tasks = [(i0, min(n_frames, i0 + step), fs, t_fft, lo, hi) for i0 in range(0, n_frames, step)]
        parts = self.pool.map(_oracle_peak_chunk, tasks)
        fi = np.concatenate([p[0] for p in parts])
        bj = np.concatenate([p[1] for p in parts])
        order = np.lexsort((fi, bj))
        return fi[order].astype(np.uint32), bj[order].astype(np.uint32)

    def rows(self, fi, bj, jobs):
        """jobs: [(fields, rows)] -> [(seconds, [row arrays])] in job order."""
        self.start({"fi": np.asarray(fi, np.uint32), "bj": np.asarray(bj, np.uint32)})
        return self.pool.map(_oracle_rows, jobs)

    def close_pool(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None
        for shm in self.shms:
            shm.close()
            shm.unlink()
        self.shms = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close_pool()


def oracle_sample_allcores(name, series, rank=0, rows_per_map=None, pool=None):
    """The oracle on every host core on a bounded sample: the full peakmap (frames split over the
    cores), then `rows_per_map` k rows of every map (rows split over the cores); the step time is
    the measured wall time with the rows extrapolated to all rows of each map."""
    from oracle import gfh_oracle as O
    spec, pm, grids = workload(name, rank)
    own = pool is None
    pool = pool or OraclePool()
    try:
        rows_per_map = rows_per_map or 4 * pool.cores
        t0 = time.perf_counter()
        fi, bj = pool.peakmap(series, spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"])
        t_pm = time.perf_counter() - t0
        jobs, updates, n_rows = [], 0, []
        for f in grids:
            og = O.make_grid(O.Grid(**{k: v for k, v in f.items() if k != "list"}))
            updates += int(((bj >= og.bin_lo) & (bj <= og.bin_hi)).sum()) * og.n_k
            rows = np.linspace(0, og.n_k - 1, min(rows_per_map, og.n_k)).astype(int)
            n_rows.append((og.n_k, rows.size))
            for chunk in np.array_split(rows, max(1, min(rows.size, pool.cores))):
                if chunk.size:
                    jobs.append((f, chunk.tolist()))
        t1 = time.perf_counter()
        pool.rows(fi, bj, jobs)
        t_rows_wall = time.perf_counter() - t1
        # wall time of the sampled rows scaled by (all rows / sampled rows), over all maps
        frac = sum(k for k, _ in n_rows) / sum(r for _, r in n_rows)
        t_step = t_pm + t_rows_wall * frac
    finally:
        if own:
            pool.close_pool()
    sample = (f"oracle peakmap of the full series ({t_pm:.1f} s, frames split over {pool.cores} "
              f"processes) + {rows_per_map} of the k rows of each of the {len(grids)} maps (rows "
              f"split over the processes, {t_rows_wall:.1f} s), extrapolated to all rows; numpy, "
              f"one thread per process")
    return updates / t_step, t_step, sample, pool.cores

def oracle_sample(name, series=None, rank=0, rows_per_map=20):
    """Times the oracle on a bounded sample: the full peakmap, then `rows_per_map` k rows of every
    map; the step time is extrapolated to all rows."""
    from oracle import gfh_oracle as O
    spec, pm, grids = workload(name, rank)
    x = spec.series() if series is None else series
    t0 = time.perf_counter()
    fi, bj = O.peakmap(x, spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"])
    t_pm = time.perf_counter() - t0
    t_rows, updates = 0.0, 0
    for f in grids:
        og = O.make_grid(O.Grid(**{k: v for k, v in f.items() if k not in ("list",)}))
        sel = (bj >= og.bin_lo) & (bj <= og.bin_hi)
        updates += int(sel.sum()) * og.n_k
        rows = np.linspace(0, og.n_k - 1, rows_per_map).astype(int)
        t1 = time.perf_counter()
        for r in rows:
            O.hough_row(og, fi, bj, int(r))
        t_rows += (time.perf_counter() - t1) * og.n_k / rows_per_map
    t_step = t_pm + t_rows
    sample = (f"oracle peakmap of the full series ({t_pm:.1f} s) + {rows_per_map} of the k rows of "
              f"each of the {len(grids)} maps, extrapolated to all rows; numpy, 1 thread")
    return updates / t_step, t_step, sample


def reference_proposer(args):
    """Reference arm of the proposer workload: the oracle's full exact Hough (the search the
    proposer prunes) on k rows of the n = 5 map of the first held-out batch, extrapolated."""
    from oracle import gfh_oracle as O
    from paper_1810_09784_gb300 import proposer as PR
    from paper_1810_09784_gb300 import synth
    spec = PR.ProposerSpec()
    s = 100011 + 30
    smp = PR.draw(spec, [s])
    inj = PR.injection_of(spec, smp, 0)
    x = synth.strain_series(int(round(spec.fs * spec.t_obs)), spec.fs, PR.series_seed(spec, s),
                            () if inj is None else (inj,))
    fi, bj = O.peakmap(x, spec.fs, spec.t_fft, spec.bin_lo, spec.bin_hi)
    o = O.make_grid(O.Grid(**{k: v for k, v in spec.grid_fields(5.0).items() if k != "list"}))
    vals = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rows = 0
        while time.perf_counter() - t0 < 2.0 and rows < o.n_k:
            O.hough_row(o, fi, bj, rows)
            rows += 1
        if i >= args.warmup:
            vals.append(fi.size * rows / (time.perf_counter() - t0))
    value = float(np.mean(vals))
    sample = (f"oracle full exact Hough, k rows of one n = 5 held-out map (its series' oracle peakmap, "
              f"{fi.size} peaks), 2 s per step, numpy, 1 thread")
    print(json.dumps({"impl": "reference", "metric": "Hough updates/s (peaks x k-bins), full-search equivalent",
                      "value": value, "unit": "updates/s", "n_gpus": args.gpus, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 2000.0, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "int32 counts, fp64 grid",
                      "data": "synthetic", "config": {"workload": "proposer (full exact search on the CPU)"},
                      "cpu_baseline": {"value": value, "unit": "updates/s", "cores": 1, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def reference_train(args):
    """Reference arm of the training workload: the oracle's network forward and backward pass
    (fp64 numpy, the kernels' bf16 storage points) on one image per step."""
    from oracle import cnn_oracle as C
    rng = np.random.default_rng(0)
    params = rng.uniform(-0.05, 0.05, C.layout()[1])
    img = C.bf16(np.log1p(rng.poisson(1.2, (1, 256, 256, 2)).astype(np.float64)))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        C.backward(C.forward(params, img), np.array([7]))
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = 1.0 / t
    cores, model = host_cpu()
    print(json.dumps({"impl": "reference", "metric": "proposal-network training images/s",
                      "value": value, "unit": "images/s", "n_gpus": args.gpus, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "fp64 (bf16 storage points)",
                      "data": "synthetic",
                      "config": {"workload": "one AdamW step of the proposal network on 256 images of 256 x 256 "
                                             "x 2 (forward, weight and input gradients, optimiser)",
                                 "batch": 256, "gflop_per_image": NET_TRAIN_FLOP / 1e9},
                      "cpu_baseline": {"value": value, "unit": "images/s", "cores": 1, "kind": "oracle",
                                       "sample": "oracle forward + backward of one image per step, numpy",
                                       "cpu_model": model, "nproc": cores},
                      "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "proposer":
        return reference_proposer(args)
    if args.workload == "followup":
        return reference_followup(args)
    if args.workload == "splice":
        return reference_splice(args)
    if args.workload == "train":
        return reference_train(args)
    from oracle import gfh_oracle as O
    spec, pm, grids = workload(args.workload, 0)
    x = spec.series()
    ogs = [O.make_grid(O.Grid(**{k: v for k, v in f.items() if k != "list"})) for f in grids]
    vals, times, walls = [], [], []
    cores, model = host_cpu()
    with OraclePool(cores) as pool:
        for i in range(args.warmup + args.steps):
            w0 = time.perf_counter()
            v, t, sample, used = oracle_sample_allcores(args.workload, x, 0, pool=pool,
                                                        rows_per_map=4 if args.workload == "paper_grids" else None)
            if i >= args.warmup:
                vals.append(v)
                times.append(t)
                walls.append(time.perf_counter() - w0)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": "Hough updates/s (peaks x k-bins)", "value": value,
            "unit": "updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32 counts, fp32 spectra, fp64 grid",
            "data": "synthetic", "config": plain_config(args.workload, spec, grids, ogs),
            "sampled_step_wall_s": float(np.mean(walls)),
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": used, "kind": "oracle",
                             "sample": sample, "cpu_model": model, "nproc": cores},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def plain_config(name, spec, grid_fields, grids):
    """The workload's `config` (the same on the GPU arm and the CPU reference arm): description,
    maps, cells, k rows and the L2 statement.  `grids` have n_x0 and n_k."""
    ld = [(g.n_x0 + 31) // 32 * 32 for g in grids]
    map_bytes = sum(g.n_k * l * 4 for g, l in zip(grids, ld))
    return {"workload": describe(name, spec, grid_fields), "maps": len(grids),
            "cells": int(sum(g.n_k * g.n_x0 for g in grids)),
            "k_rows": sorted({int(g.n_k) for g in grids}),
            "l2": "inputs larger than L2 (series %d MB, maps %d MB per step)"
                  % (spec.n_samples * 4 // 1000000, map_bytes // 1000000)}


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------

def run_gpu(args):
    import torch

    from paper_1810_09784_gb300 import build as _build
    from paper_1810_09784_gb300 import gfh

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    # the library works on its own stream (also the graph-capture stream)
    stream = torch.cuda.Stream()
    ctx = gfh.Context(local, stream)

    spec, pm, grid_fields = workload(args.workload, rank)
    if args.maps and args.maps < len(grid_fields):
        keep = np.linspace(0, len(grid_fields) - 1, args.maps).round().astype(int)
        grid_fields = [grid_fields[i] for i in sorted(set(keep))]
    if args.only_n is not None:
        grid_fields = [f for f in grid_fields if abs(f["n"] - args.only_n) < 1e-9]
        if not grid_fields:
            raise SystemExit(f"no map with n = {args.only_n}")
    series_np = spec.series()
    x_host = torch.from_numpy(series_np).pin_memory()
    x_dev = x_host.cuda()
    grids = [gfh.grid_make(gfh.Grid(**f)) for f in grid_fields]
    maps = [torch.empty((g.n_k, g.ld_x0), dtype=torch.int32, device="cuda") for g in grids]
    cands = [torch.empty(g.n_bands * gfh.CANDIDATE_BYTES, dtype=torch.uint8, device="cuda") for g in grids]
    stats = torch.empty(len(grids) * gfh.STATS_BYTES, dtype=torch.uint8, device="cuda")
    cand_host = [torch.empty_like(c, device="cpu").pin_memory() for c in cands]
    tile = tuple(int(v) for v in args.tile.split(",")) if args.tile else None
    t_plan = time.perf_counter()
    plan = gfh.Plan(ctx, grids, maps, cands, stats, tile=tile)
    t_plan = time.perf_counter() - t_plan
    cap = int(spec.n_fft * (pm["bin_hi"] - pm["bin_lo"] + 1) * 0.12) + 1024
    fo = torch.empty(cap, dtype=torch.int32, device="cuda")
    bo = torch.empty(cap, dtype=torch.int32, device="cuda")
    off = torch.zeros(2, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()

    def step(h2d=False, stage_events=None):
        """One search step through the public API (the peakmap count comes back to the host)."""
        if h2d:
            x_dev.copy_(x_host, non_blocking=True)
        n = ctx.peakmap(x_dev, spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"], 2.5, fo, bo)
        off[1] = n
        if stage_events is not None:
            stage_events[0].record(stream)
        plan.execute(fo, bo, off, 1)
        if stage_events is not None:
            stage_events[1].record(stream)
        if h2d:
            for c, h in zip(cands, cand_host):
                h.copy_(c, non_blocking=True)
        return n

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            n_peaks = step()
        torch.cuda.synchronize()
        if ctx.check() != gfh.GFH_OK:
            raise RuntimeError("input check failed")
        tuned, t_tune = None, 0.0
        if not args.no_autotune and tile is None:
            t_tune = time.perf_counter()
            tuned, _ = plan.autotune(fo, bo, off, 1, reps=2)
            t_tune = time.perf_counter() - t_tune
            step()
            torch.cuda.synchronize()
    # updates of this rank's step: peaks inside each map's band x its k rows
    bins = bo[:n_peaks].cpu().numpy()
    updates = sum(int(((bins >= g.bin_lo) & (bins <= g.bin_hi)).sum()) * g.n_k for g in grids)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def reduce(v, op):
        if world == 1:
            return v
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=op)
        return float(t.item())

    import torch.distributed as tdist
    MAX, SUM = (tdist.ReduceOp.MAX, tdist.ReduceOp.SUM) if world > 1 else (None, None)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    # ---- CUDA graph of the whole step: asynchronous peakmap + plan, no host round trip
    graph = None
    if not args.no_graph:
        with torch.cuda.stream(stream):
            ctx.peakmap_async(x_dev, spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"], 2.5, fo, bo, off[1:2])
            plan.execute(fo, bo, off, 1)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            ctx.peakmap_async(x_dev, spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"], 2.5, fo, bo, off[1:2])
            plan.execute(fo, bo, off, 1)
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        if ctx.check() != gfh.GFH_OK or int(off[1].item()) != n_peaks:
            raise RuntimeError("graph replay differs from the direct step")

    # ---- device-resident timing (clocks sampled meanwhile)
    sampler = ClockSampler(local)
    with sampler, torch.cuda.stream(stream):
        barrier()
        a, b = ev(), ev()
        hough = [(ev(), ev()) for _ in range(args.steps)]
        a.record(stream)
        for i in range(args.steps):
            step(stage_events=hough[i])
        b.record(stream)
        barrier()
        ms_direct = a.elapsed_time(b) / args.steps
        ms_graph = None
        if graph is not None:
            barrier()
            torch.cuda.nvtx.range_push("timed_steps")       # lets a profiler select these launches
            a.record(stream)
            for _ in range(args.steps):
                graph.replay()
            b.record(stream)
            barrier()
            torch.cuda.nvtx.range_pop()
            ms_graph = a.elapsed_time(b) / args.steps
    clocks = sampler.summary()
    ms_hough = sum(e0.elapsed_time(e1) for e0, e1 in hough) / args.steps
    ms = ms_graph if ms_graph is not None else ms_direct
    ms_max, total_updates = ranks.combine(ms, float(updates), device="cuda")
    value = total_updates / (ms_max * 1e-3)

    # ---- end to end through the public API with host buffers: every step copies its series from
    # pinned host memory and reads its candidates back; the copy of step i + 1 (second device
    # buffer, copy stream) overlaps the search of step i, as a streaming pipeline would
    x_buf = [x_dev, torch.empty_like(x_dev)]
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]

    h2d_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]

    def e2e_step(i, timed=False):
        k = i & 1
        copy_stream.wait_event(consumed[k])              # buffer k no longer read
        if timed:
            h2d_ev[i][0].record(copy_stream)
        with torch.cuda.stream(copy_stream):
            x_buf[k].copy_(x_host, non_blocking=True)
        copied[k].record(copy_stream)
        if timed:
            h2d_ev[i][1].record(copy_stream)
        stream.wait_event(copied[k])
        with torch.cuda.stream(stream):
            ctx.peakmap_async(x_buf[k], spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"], 2.5, fo, bo,
                              off[1:2])
            plan.execute(fo, bo, off, 1)
            for c, h in zip(cands, cand_host):
                h.copy_(c, non_blocking=True)
        consumed[k].record(stream)

    for i in range(max(args.warmup, 2)):                # untimed: both buffers used once
        e2e_step(i)
    barrier()
    a.record(stream)
    copy_stream.wait_event(a)
    for i in range(args.steps):
        e2e_step(i, timed=True)
    b.record(stream)
    barrier()
    ms_e2e = reduce(a.elapsed_time(b) / args.steps, MAX)
    ms_h2d = sum(e0.elapsed_time(e1) for e0, e1 in h2d_ev) / args.steps
    if ctx.check() != gfh.GFH_OK or int(off[1].item()) != n_peaks:
        raise RuntimeError("end-to-end steps differ from the direct step")
    h2d = x_host.numel() * 4
    d2h = sum(c.numel() for c in cands)

    # ---- batched vs one plan per map (the maps share the step's peak list)
    sequential = None
    if args.workload in ("batched_n", "paper_grids") or len(grids) > 1 and args.sequential:
        cfg = tuned or tile
        singles = [gfh.Plan(ctx, [g], [m], [c], None, tile=cfg) for g, m, c in zip(grids, maps, cands)]
        with torch.cuda.stream(stream):
            for sp in singles:
                sp.execute(fo, bo, off, 1)
            barrier()
            a.record(stream)
            for _ in range(args.steps):
                for sp in singles:
                    sp.execute(fo, bo, off, 1)
            b.record(stream)
            barrier()
        ms_seq = a.elapsed_time(b) / args.steps
        sequential = {"ms_hough_one_plan_per_map": ms_seq, "ms_hough_batched": ms_hough,
                      "speedup": ms_seq / ms_hough}
        for sp in singles:
            sp.close()

    # ---- the paper's squares selector (Sec. IV) on every map of the step, 5 x 5 squares
    squares = None
    if args.workload == "plain_paper":
        sq_out = [torch.empty(2 * 25 * gfh.CANDIDATE_BYTES, dtype=torch.uint8, device="cuda") for _ in grids]
        with torch.cuda.stream(stream):
            for g, m, o in zip(grids, maps, sq_out):
                ctx.select_squares(m, g, 5, 5, o)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for g, m, o in zip(grids, maps, sq_out):
                ctx.select_squares(m, g, 5, 5, o)
            torch.cuda.synchronize()
            ms_sq = (time.perf_counter() - t0) * 1e3
        ana_bytes = 0
        for g in grids:
            band = gfh.grid_columns(g)[0]
            ana_bytes += int((band >= 0).sum()) * g.n_k * 4
        squares = {"maps": len(grids), "squares_per_map": 25, "ms_all_maps": ms_sq,
                   "timing": "host wall clock around the synchronous calls (scratch allocation included)",
                   "analysis_cells_bytes_read": ana_bytes,
                   "achieved_gbs": ana_bytes / (ms_sq * 1e-3) / 1e9, "hbm_peak_gbs": HBM_PEAK}
    if rank != 0:
        plan.close()
        ctx.close()
        return
    atomics = 2.0 * updates
    achieved = atomics / (ms_hough * 1e-3) / 1e9
    map_bytes = sum(g.n_k * g.ld_x0 * 4 for g in grids)
    line = {
        "metric": "Hough updates/s (peaks x k-bins)", "value": value, "unit": "updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32 counts, fp32 spectra, fp64 grid", "data": "synthetic",
        "config": plain_config(args.workload, spec, grid_fields, grids),
        "work": {"peaks": n_peaks, "updates_per_step": updates},
        "run": {"tile": list(tile) if tile else (list(tuned) if tuned else "default"),
                "tile_source": "given" if tile else ("autotuned" if tuned else "default"),
                "timing": "CUDA graph of the step" if graph is not None else "direct calls",
                "plan_build_s": round(t_plan, 3), "autotune_s": round(t_tune, 3)},
        "breakdown_ms": {"step_graph": ms_graph, "step_direct": ms_direct, "hough_select": ms_hough,
                         "peakmap_and_host": ms_direct - ms_hough},
        "roofline": {**atomic_roofline(ctx, stream, achieved),
                     "traffic": traffic_for("k_hough") if args.workload == "plain_paper" and not args.maps else None,
                     "issue": issue_roofline(updates / (ms_hough * 1e-3), atomic_peak(ctx, stream)[1]["sms"],
                                             (clocks or {}).get("sm_mhz") or 2070.0)
                     if args.workload == "plain_paper" and not args.maps else None,
                     "hbm": {"map_store_bytes": map_bytes, "achieved_gbs": map_bytes / (ms_hough * 1e-3) / 1e9,
                             "peak_gbs": HBM_PEAK, "frac": map_bytes / (ms_hough * 1e-3) / 1e9 / HBM_PEAK,
                             "peak_source": HBM_PEAK_SRC}},
        "e2e": {"value": total_updates / (ms_e2e * 1e-3), "unit": "updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
                "h2d_ms_per_copy": ms_h2d, "h2d_gbs": h2d / (ms_h2d * 1e-3) / 1e9,
                "timing": "asynchronous public calls after untimed warm-up steps; each step's "
                          "series copied from pinned host memory on a copy stream into one of two "
                          "device buffers (overlapping the previous step's search) and its "
                          "candidates read back"},
        "squares_selector": squares,
        "gpu_launches": 9 * args.steps,
        "clocks": clocks,
    }
    if sequential:
        line["batched_vs_one_plan_per_map"] = sequential
    if args.workload == "plain_paper" and world == 1 and not args.no_extras:
        # configs 3-5 as compact sub-objects of the default line (their own timed regions)
        ext_steps, ext_warm = max(3, min(args.steps, 10)), max(3, args.warmup)
        t0 = time.perf_counter()
        line["batched_n"] = measure_batched_n(ctx, stream, ext_steps, ext_warm)
        line["uneven"] = measure_uneven(ctx, stream, ext_steps, ext_warm)
        line["proposer"] = measure_proposer(ctx, stream, ext_steps, ext_warm, eval_maps=args.eval_maps)
        line["extras_s"] = round(time.perf_counter() - t0, 1)
    if world == 1 and not args.no_cpu_baseline:
        cores, model = host_cpu()
        v, t, sample, used = oracle_sample_allcores(args.workload, series_np,
                                                    rows_per_map=4 if args.workload == "paper_grids" else None)
        v1, t1, sample1 = oracle_sample(args.workload, series_np, rows_per_map=2 if args.workload == "paper_grids" else 5)
        line["cpu_baseline"] = {"value": v, "unit": "updates/s", "cores": used, "kind": "oracle",
                                "sample": sample, "cpu_model": model, "nproc": cores,
                                "one_core": {"value": v1, "sample": sample1}}
    print(json.dumps(line), flush=True)
    plan.close()
    ctx.close()


# ---------------------------------------------------------------------------------------------
# Compact measurements of the batched and pruned forms (sub-objects of the default line)
# ---------------------------------------------------------------------------------------------

def _time_ms(stream, fn, steps):
    """Mean device time of fn() over `steps` calls, CUDA events on `stream`."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def _roofline_of(ctx, stream, updates, map_bytes, ms):
    """The accumulator's bound: max(map store / HBM peak, 2 atomics per update / atomic peak)."""
    peak, _ = atomic_peak(ctx, stream)
    t_atomic = 2.0 * updates / (peak * 1e9) * 1e3
    t_hbm = map_bytes / (HBM_PEAK * 1e9) * 1e3
    bound = "smem_atomic" if t_atomic >= t_hbm else "hbm"
    return {"bound": bound, "ms_at_bound": max(t_atomic, t_hbm), "frac": max(t_atomic, t_hbm) / ms,
            "atomic_ms": t_atomic, "hbm_ms": t_hbm, "atomic_peak_gatomic_s": peak,
            "hbm_peak_gbs": HBM_PEAK}


def measure_batched_n(ctx, stream, steps, warmup, tile=(16, 3072, 1024, 1)):
    """Config 3: the plain_small peakmap at 51 braking indices, one launch (CUDA graph), against
    one plan per braking index run one after another.  The tile draws one form per warp (form 1):
    measured 20.3 ms against 21.1 ms with each peak in its own form, maps identical (the tall
    low-n maps mix interior and edge peaks in many warps)."""
    import torch
    from paper_1810_09784_gb300 import gfh
    spec, pm, grid_fields = workloads.batched_n(seed=ranks.rank_seed(1, 0))
    x = torch.from_numpy(spec.series()).cuda()
    cap = int(spec.n_fft * (pm["bin_hi"] - pm["bin_lo"] + 1) * 0.12) + 1024
    fo = torch.empty(cap, dtype=torch.int32, device="cuda")
    bo = torch.empty(cap, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        n = ctx.peakmap(x, spec.fs, spec.t_fft, pm["bin_lo"], pm["bin_hi"], 2.5, fo, bo)
    off = torch.tensor([0, n], dtype=torch.int64, device="cuda")
    grids = [gfh.grid_make(gfh.Grid(**f)) for f in grid_fields]
    bins = bo[:n].cpu().numpy()
    updates = sum(int(((bins >= g.bin_lo) & (bins <= g.bin_hi)).sum()) * g.n_k for g in grids)
    maps = [torch.empty((g.n_k, g.ld_x0), dtype=torch.int32, device="cuda") for g in grids]
    cands = [torch.empty(g.n_bands * gfh.CANDIDATE_BYTES, dtype=torch.uint8, device="cuda") for g in grids]
    stats = torch.empty(len(grids) * gfh.STATS_BYTES, dtype=torch.uint8, device="cuda")
    plan = gfh.Plan(ctx, grids, maps, cands, stats, tile=tile)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            plan.execute(fo, bo, off, 1)
        torch.cuda.synchronize()
        if ctx.check() != gfh.GFH_OK:
            raise RuntimeError("batched_n: input check failed")
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            plan.execute(fo, bo, off, 1)
        graph.replay()
        ms = _time_ms(stream, graph.replay, steps)
        singles = [gfh.Plan(ctx, [g], [m], [c], None, tile=tile) for g, m, c in zip(grids, maps, cands)]
        for sp in singles:
            sp.execute(fo, bo, off, 1)
        ms_seq = _time_ms(stream, lambda: [sp.execute(fo, bo, off, 1) for sp in singles], max(2, steps // 4))
    for sp in singles:
        sp.close()
    map_bytes = sum(g.n_k * g.ld_x0 * 4 for g in grids)
    out = {"workload": "batched_n: the plain_small peakmap at n = 2.0..7.0 (51 maps, 4000 -> 1000 "
                       "k rows), one launch replayed as a CUDA graph",
           "maps": len(grids), "peaks": int(n), "updates_per_step": updates,
           "map_bytes": map_bytes, "tile": list(tile), "ms_per_step": ms,
           "updates_per_s": updates / (ms * 1e-3), "ms_one_plan_per_map": ms_seq,
           "speedup_vs_one_plan_per_map": ms_seq / ms,
           "roofline": _roofline_of(ctx, stream, updates, map_bytes, ms)}
    plan.close()
    del maps, cands, stats, graph
    torch.cuda.empty_cache()
    return out


def measure_uneven(ctx, stream, steps, warmup, tile=(16, 3072, 1024)):
    """Config 4: 256 uneven peakmaps (statistical model), every sub-band map in one launch, against
    one plan per peakmap run one after another."""
    import torch
    from paper_1810_09784_gb300 import gfh
    t0 = time.perf_counter()
    lists, grid_fields, _ = workloads.uneven(seed=ranks.rank_seed(4, 0))
    t_gen = time.perf_counter() - t0
    off_np = np.cumsum([0] + [len(f) for f, _ in lists]).astype(np.int64)
    fi = torch.from_numpy(np.concatenate([f for f, _ in lists]).view(np.int32)).cuda()
    bj = torch.from_numpy(np.concatenate([b for _, b in lists]).view(np.int32)).cuda()
    off = torch.from_numpy(off_np).cuda()
    grids = [gfh.grid_make(gfh.Grid(**f)) for f in grid_fields]
    updates = 0
    for f, g in zip(grid_fields, grids):
        b = lists[f["list"]][1]
        updates += int(((b >= g.bin_lo) & (b <= g.bin_hi)).sum()) * g.n_k
    del lists
    maps = [torch.empty((g.n_k, g.ld_x0), dtype=torch.int32, device="cuda") for g in grids]
    cands = [torch.empty(g.n_bands * gfh.CANDIDATE_BYTES, dtype=torch.uint8, device="cuda") for g in grids]
    stats = torch.empty(len(grids) * gfh.STATS_BYTES, dtype=torch.uint8, device="cuda")
    plan = gfh.Plan(ctx, grids, maps, cands, stats, tile=tile)
    nl = len(off_np) - 1
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            plan.execute(fi, bj, off, nl)
        torch.cuda.synchronize()
        if ctx.check() != gfh.GFH_OK:
            raise RuntimeError("uneven: input check failed")
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            plan.execute(fi, bj, off, nl)
        graph.replay()
        ms = _time_ms(stream, graph.replay, steps)
        per_list = {}
        for gf, g, m, c in zip(grid_fields, grids, maps, cands):
            per_list.setdefault(gf["list"], []).append((g, m, c))
        singles = [gfh.Plan(ctx, [x[0] for x in v], [x[1] for x in v], [x[2] for x in v], None,
                            tile=tile) for v in per_list.values()]
        for sp in singles:
            sp.execute(fi, bj, off, nl)
        ms_seq = _time_ms(stream, lambda: [sp.execute(fi, bj, off, nl) for sp in singles], 1)
    for sp in singles:
        sp.close()
    map_bytes = sum(g.n_k * g.ld_x0 * 4 for g in grids)
    npk = np.diff(off_np)
    out = {"workload": "uneven: 256 statistical peakmaps (1-24 h, T_FFT 1-8 s, bands inside "
                       "50-2000 Hz, 0-3 power-law tracks each), 100 Hz sub-bands, 1000 k rows, "
                       "every map in one launch replayed as a CUDA graph",
           "data": "statistical peakmap model (independent cells at p0, tracks at p = 0.6)",
           "peakmaps": nl, "maps": len(grids), "peaks": int(off_np[-1]),
           "peaks_per_peakmap": [int(npk.min()), int(npk.max())], "updates_per_step": updates,
           "map_bytes": map_bytes, "tile": list(tile), "generate_s": round(t_gen, 1),
           "ms_per_step": ms, "updates_per_s": updates / (ms * 1e-3),
           "ms_one_plan_per_peakmap": ms_seq, "speedup_vs_one_plan_per_peakmap": ms_seq / ms,
           "roofline": _roofline_of(ctx, stream, updates, map_bytes, ms)}
    plan.close()
    del maps, cands, stats, graph, fi, bj
    torch.cuda.empty_cache()
    return out


def measure_proposer(ctx, stream, steps, warmup, eval_maps=51 * 196):
    """Config 5 from the committed checkpoint (no training here): recall of the pruned search
    against the full exact Hough on held-out maps built from seeded series through gfh_peakmap,
    and the time of one batch of 51 maps (resident peak lists) searched in full and pruned, for
    the network and for the non-learned line-sum ranker."""
    import torch
    from paper_1810_09784_gb300 import gfh
    from paper_1810_09784_gb300 import proposer as PR
    spec = PR.ProposerSpec()
    nl = len(PR.N_GRID)
    path = PR.checkpoint_path()
    state, meta = PR.load_checkpoint(path)
    out = {"workload": "proposer: 51 maps per step (n = 2.0..7.0), plain_small-shaped (1799 FFTs, "
                       "100-400 Hz, 500 k rows), half with one power-law injection (SNR 2-8); "
                       "at most 32 of 64 x 64 coarse tiles per map, full search of maps whose "
                       "proposal leaves more than tau",
           "data": "peakmaps built by gfh_peakmap from seeded white-noise series with power-law "
                   "injections",
           "checkpoint": f"{path.parent.name}/{path.name}: trained on {meta.get('n_train')} "
                         f"series peakmaps, {meta.get('epochs')} passes, step {state['step']}"}
    with torch.cuda.stream(stream):
        net = gfh.Cnn(ctx, nl, seed=1)
        net.set_state(state)
        bank = PR.HoughBank(ctx, spec, max_sel=256)
        bank.load_peaks(PR.draw(spec, np.arange(PR.VALIDATION_FIRST, PR.VALIDATION_FIRST + nl)))
        tuned, _ = bank.autotune()
        hm = meta.get("heuristic", {})
        heur = PR.LineHeuristic(ctx, spec, hm.get("beta", 1.0), hm.get("det_a", 1.0), hm.get("det_b", 6.0))
        scorers = {f"{name}_{cap}": (sc, meta["tau"][key][str(cap)], cap)
                   for cap in (32, 256)
                   for name, key, sc in (("network", "network", net), ("line_heuristic", "heuristic", heur))}
        for name, (sc, tau, cap) in scorers.items():
            t0 = time.perf_counter()
            summ = PR.summarize(PR.evaluate(ctx, sc, spec, PR.HELD_OUT_FIRST, eval_maps, bank, tau, cap))
            search = PR.PrunedSearch(ctx, sc, bank, tau, cap)
            t_full, t_pr, upd = [], [], []
            for st in range(warmup + steps):
                s0 = PR.HELD_OUT_FIRST + nl * st
                bank.load_peaks(PR.draw(spec, np.arange(s0, s0 + nl)))
                torch.cuda.synchronize()
                timed = st >= warmup
                if timed:
                    torch.cuda.nvtx.range_push("full_exact")
                a = _time_ms(stream, bank.full, 1)
                if timed:
                    torch.cuda.nvtx.range_pop()
                    torch.cuda.nvtx.range_push(f"pruned_{name}")
                b = _time_ms(stream, search.run, 1)
                if timed:
                    torch.cuda.nvtx.range_pop()
                    t_full.append(a)
                    t_pr.append(b)
                    upd.append(bank.updates())
            ms_full, ms_pr = float(np.mean(t_full)), float(np.mean(t_pr))
            out[name] = {"tiles_at_most": cap, "tau": tau, "recall": summ["recall"],
                         "held_out_maps": summ["maps"],
                         "detected_full": summ["det_full"], "detected_kept": summ["det_kept"],
                         "fallback_frac": summ["fallback_frac"],
                         "fallback_noise": summ["fallback_noise"],
                         "mean_tiles_pruned": summ["mean_tiles_pruned"],
                         "ms_full_exact_per_step": ms_full, "ms_pruned_per_step": ms_pr,
                         "speedup_vs_full_exact": ms_full / ms_pr,
                         "full_search_updates_per_step": float(np.mean(upd)),
                         "eval_s": round(time.perf_counter() - t0, 1)}
        out["tile"] = list(tuned)
        out["line_heuristic_parameters"] = {"beta": heur.beta, "det_a": heur.det_a, "det_b": heur.det_b}
        ok = [k for k in out if k.startswith("network_") and out[k]["recall"] >= 0.99]
        best = max(ok, key=lambda k: out[k]["speedup_vs_full_exact"]) if ok else None
        out["speedup_vs_full_exact"] = out[best]["speedup_vs_full_exact"] if best else None
        out["recall"] = out[best]["recall"] if best else None
        out["operating_point"] = best
        f0_, f1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        search = PR.PrunedSearch(ctx, net, bank, meta["tau"]["network"]["32"], 32)
        search.propose()
        torch.cuda.synchronize()
        out["network_forward_ms_51_maps"] = _time_ms(stream, lambda: net.forward(search.images, search.logits), 5)
    net.close()
    bank.plan.close()
    torch.cuda.empty_cache()
    return out


# multiply-adds per image of the proposal network: forward of the five 3x3 layers, their weight
# gradients (the same count) and the input gradients of layers 2-5
_NET_MACS = [256 * 256 * 32 * 18, 128 * 128 * 32 * 288, 128 * 128 * 64 * 288, 64 * 64 * 64 * 576,
             64 * 64 * 64 * 576]
NET_FWD_FLOP = 2.0 * sum(_NET_MACS)
NET_TRAIN_FLOP = 2.0 * (2 * sum(_NET_MACS) + sum(_NET_MACS[1:]))
# kernels one AdamW step launches: forward the image padded to 8 channels, 5 convolutions, pool,
# head, softmax/CE; backward the head (weights, chunk sum, input), 4 input gradients, 5 weight
# gradients (bias sums inside) with their weight and bias chunk sums; optimiser, then 5 bf16
# weight copies
TRAIN_LAUNCHES = 9 + 3 + 4 + 5 * 3 + 1 + 5


def run_train(args):
    """Training step of the proposal network: one AdamW step on a batch of 256 images (forward,
    every gradient, optimiser), timed with CUDA events over `steps` steps on resident images."""
    import torch
    from paper_1810_09784_gb300 import build as _build
    from paper_1810_09784_gb300 import gfh
    from paper_1810_09784_gb300 import proposer as PR
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    stream = torch.cuda.Stream()
    ctx = gfh.Context(local, stream)
    spec = PR.ProposerSpec()
    B = args.batch
    with torch.cuda.stream(stream):
        cache = PR.ImageCache(ctx, spec, 0, 2 * B)
        net = gfh.Cnn(ctx, B, seed=1)
        for i in range(args.warmup):
            im, lb = cache.batch((i % 2) * B, B)
            net.train_step(im, lb, 1e-3, 1e-4, want_loss=False)
        torch.cuda.synchronize()
        if ctx.check() != gfh.GFH_OK:
            raise RuntimeError("training step flagged an error")
        sampler = ClockSampler(local)
        with sampler:
            torch.cuda.nvtx.range_push("timed_steps")
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for i in range(args.steps):
                im, lb = cache.batch((i % 2) * B, B)
                net.train_step(im, lb, 1e-3, 1e-4, want_loss=False)
            b.record(stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        ms = a.elapsed_time(b) / args.steps
        fw = _time_ms(stream, lambda: net.forward(cache.images[:B]), max(3, args.steps))
    net.close()
    if rank != 0:
        return
    peak = PEAKS.get("bf16_tflops_sustained")
    tflops = NET_TRAIN_FLOP * B / (ms * 1e-3) / 1e12
    fw_tflops = NET_FWD_FLOP * B / (fw * 1e-3) / 1e12
    print(json.dumps({
        "metric": "proposal-network training images/s", "value": B / (ms * 1e-3), "unit": "images/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 weights and activations, fp32 accumulate", "data": "synthetic (series peakmaps)",
        "config": {"workload": f"one AdamW step of the proposal network on {B} images of 256 x 256 "
                               "x 2 (forward, weight and input gradients, optimiser)",
                   "batch": B, "gflop_per_image": NET_TRAIN_FLOP / 1e9},
        "roofline": {"bound": "tensor", "kernel": "whole training step", "achieved": tflops,
                     "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak if peak else None,
                     "peak_source": "measured cuBLAS bf16, sustained" if peak else "none",
                     "algorithmic": f"{NET_TRAIN_FLOP / 1e9:.2f} GFLOP per image", "traffic": None},
        "forward": {"ms_batch": fw, "tflops": fw_tflops,
                    "frac_of_burst_peak": fw_tflops / PEAKS["bf16_tflops"] if "bf16_tflops" in PEAKS else None},
        "gpu_launches": TRAIN_LAUNCHES * args.steps, "clocks": sampler.summary()}), flush=True)
    ctx.close()


def run_gpu_lists(args):
    """Peak-list workload (uneven): a step is the batched Hough + selection of every sub-band map
    of every peakmap, in one launch (replayed as a CUDA graph)."""
    import torch

    from paper_1810_09784_gb300 import build as _build
    from paper_1810_09784_gb300 import gfh

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    stream = torch.cuda.Stream()
    ctx = gfh.Context(local, stream)
    t_gen = time.perf_counter()
    lists, grid_fields, specs = workloads.uneven(seed=ranks.rank_seed(4, rank))
    t_gen = time.perf_counter() - t_gen
    off_np = np.cumsum([0] + [len(f) for f, _ in lists]).astype(np.int64)
    fi_host = torch.from_numpy(np.concatenate([f for f, _ in lists]).view(np.int32)).pin_memory()
    bj_host = torch.from_numpy(np.concatenate([b for _, b in lists]).view(np.int32)).pin_memory()
    fi, bj = fi_host.cuda(), bj_host.cuda()
    off = torch.from_numpy(off_np).cuda()
    grids = [gfh.grid_make(gfh.Grid(**f)) for f in grid_fields]
    maps = [torch.empty((g.n_k, g.ld_x0), dtype=torch.int32, device="cuda") for g in grids]
    cands = [torch.empty(g.n_bands * gfh.CANDIDATE_BYTES, dtype=torch.uint8, device="cuda") for g in grids]
    stats = torch.empty(len(grids) * gfh.STATS_BYTES, dtype=torch.uint8, device="cuda")
    tile = tuple(int(v) for v in args.tile.split(",")) if args.tile else None
    t_plan = time.perf_counter()
    plan = gfh.Plan(ctx, grids, maps, cands, stats, tile=tile)
    t_plan = time.perf_counter() - t_plan
    updates = 0
    for f, g in zip(grid_fields, grids):
        b = lists[f["list"]][1]
        updates += int(((b >= g.bin_lo) & (b <= g.bin_hi)).sum()) * g.n_k
    ev = lambda: torch.cuda.Event(enable_timing=True)
    a, b_ = ev(), ev()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.execute(fi, bj, off, len(lists))
        torch.cuda.synchronize()
        if ctx.check() != gfh.GFH_OK:
            raise RuntimeError("input check failed")
        graph = None
        if not args.no_graph:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                plan.execute(fi, bj, off, len(lists))
            graph.replay()
            torch.cuda.synchronize()
        sampler = ClockSampler(local)
        with sampler:
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(args.steps):
                if graph is not None:
                    graph.replay()
                else:
                    plan.execute(fi, bj, off, len(lists))
            b_.record(stream)
            torch.cuda.synchronize()
        ms = a.elapsed_time(b_) / args.steps
        clocks = sampler.summary()
        # end to end: peak lists from pinned host memory, candidates back to the host
        cand_host = [torch.empty_like(c, device="cpu").pin_memory() for c in cands]
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            fi.copy_(fi_host, non_blocking=True)
            bj.copy_(bj_host, non_blocking=True)
            plan.execute(fi, bj, off, len(lists))
            for c, h in zip(cands, cand_host):
                h.copy_(c, non_blocking=True)
        b_.record(stream)
        torch.cuda.synchronize()
        ms_e2e = ranks.combine(a.elapsed_time(b_) / args.steps, 0.0, device="cuda")[0]
        # one plan per peakmap, executed one after another
        per_list = {}
        for gf, g, m, c in zip(grid_fields, grids, maps, cands):
            per_list.setdefault(gf["list"], []).append((g, m, c))
        singles = [gfh.Plan(ctx, [x[0] for x in v], [x[1] for x in v], [x[2] for x in v], None,
                            tile=tile) for v in per_list.values()]
        for sp in singles:
            sp.execute(fi, bj, off, len(lists))
        torch.cuda.synchronize()
        a.record(stream)
        for sp in singles:
            sp.execute(fi, bj, off, len(lists))
        b_.record(stream)
        torch.cuda.synchronize()
        ms_seq = a.elapsed_time(b_)
        for sp in singles:
            sp.close()
    ms_max, total = ranks.combine(ms, float(updates), device="cuda")
    if rank == 0:
        map_bytes = sum(g.n_k * g.ld_x0 * 4 for g in grids)
        achieved = 2.0 * updates / (ms * 1e-3) / 1e9
        npk = np.diff(off_np)
        line = {
            "metric": "Hough updates/s (peaks x k-bins)", "value": total / (ms_max * 1e-3),
            "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32 counts, fp64 grid", "data": "synthetic (statistical peakmap model)",
            "config": {"workload": "uneven: 256 independent peakmaps, 1-24 h, T_FFT 1-8 s, bands "
                                   "inside 50-2000 Hz, 0-3 power-law injections each; 100 Hz "
                                   "sub-bands (+50 Hz), 1000 k rows; all maps in one launch",
                       "peakmaps": len(lists), "maps": len(grids), "peaks": int(off_np[-1]),
                       "peaks_per_peakmap": [int(npk.min()), int(npk.max())],
                       "updates_per_step": updates, "cells": int(sum(g.n_k * g.n_x0 for g in grids)),
                       "l2": "inputs larger than L2 (%d MB of peaks, %d MB of maps)" % (off_np[-1] * 8 // 1000000, map_bytes // 1000000),
                       "tile": list(tile) if tile else "default", "timing": "CUDA graph" if graph is not None else "direct",
                       "generate_s": round(t_gen, 2), "plan_build_s": round(t_plan, 2)},
            "roofline": {**atomic_roofline(ctx, stream, achieved), "traffic": None,
                         "hbm": {"map_store_bytes": map_bytes, "achieved_gbs": map_bytes / (ms * 1e-3) / 1e9,
                                 "peak_gbs": HBM_PEAK, "frac": map_bytes / (ms * 1e-3) / 1e9 / HBM_PEAK}},
            "e2e": {"value": total / (ms_e2e * 1e-3), "unit": "updates/s",
                    "h2d_bytes_per_step": int(off_np[-1]) * 8, "d2h_bytes_per_step": sum(c.numel() for c in cands),
                    "ms_per_step": ms_e2e},
            "batched_vs_one_plan_per_peakmap": {"ms_one_plan_per_peakmap": ms_seq, "ms_batched": ms,
                                                "speedup": ms_seq / ms},
            "gpu_launches": 4 * args.steps, "clocks": clocks}
        print(json.dumps(line), flush=True)
    plan.close()
    ctx.close()


def run_proposer(args):
    """Learned proposer + exact Hough, from the committed checkpoint (the network was trained on the
    GPU by the library's kernels: `python -m paper_1810_09784_gb300.proposer train`).  A step is one
    batch of 51 held-out maps (one per braking index) with resident peak lists, searched by the full
    exact Hough and by the pruned search (images, network, proposals, one exact-Hough launch over the
    proposed tiles and over every map whose proposal cannot reach tau), at both tile budgets, for
    the network and for the non-learned line ranker; recall on 9,996 held-out series maps."""
    import torch

    from paper_1810_09784_gb300 import build as _build
    from paper_1810_09784_gb300 import gfh

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    stream = torch.cuda.Stream()
    ctx = gfh.Context(local, stream)
    sampler = ClockSampler(local)
    with sampler:
        res = measure_proposer(ctx, stream, args.steps, args.warmup, eval_maps=args.eval_maps)
    if rank != 0:
        return
    op = res[res["operating_point"]] if res["operating_point"] else res["network_32"]
    value = op["full_search_updates_per_step"] / (op["ms_pruned_per_step"] * 1e-3)
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import gfh_oracle as O
        from paper_1810_09784_gb300 import proposer as PR
        spec = PR.ProposerSpec()
        src = PR.PeakSource(ctx, spec, 51)
        with torch.cuda.stream(stream):
            src.load(PR.draw(spec, np.arange(PR.HELD_OUT_FIRST, PR.HELD_OUT_FIRST + 51)))
        o0, o1 = src.offs_host[30], src.offs_host[31]           # the n = 5 map
        fi = src.fft_c[o0:o1].cpu().numpy().view(np.uint32)
        bj = src.bin_c[o0:o1].cpu().numpy().view(np.uint32)
        og = O.make_grid(O.Grid(**{k: v for k, v in spec.grid_fields(5.0).items() if k != "list"}))
        t0 = time.perf_counter()
        rows = 0
        while time.perf_counter() - t0 < 10.0 and rows < og.n_k:
            O.hough_row(og, fi, bj, rows)
            rows += 1
        dt = time.perf_counter() - t0
        cpu = {"value": fi.size * rows / dt, "unit": "updates/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle full exact Hough of {rows} k rows of the n = 5 map of one held-out "
                         f"batch ({fi.size} peaks), numpy, 1 thread"}
    line = {
        "metric": "Hough updates/s (peaks x k-bins), full-search equivalent", "value": value,
        "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": op["ms_pruned_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32 counts; bf16 network, fp32 accumulate",
        "data": res["data"], "config": {"workload": res["workload"], "checkpoint": res["checkpoint"]},
        "proposer": res, "speedup_vs_full_exact": res["speedup_vs_full_exact"],
        "recall": res["recall"], "operating_point": res["operating_point"],
        "roofline": {"bound": "tensor", "kernel": "network forward (k_conv_fwd_tc, 5 layers)",
                     "achieved": NET_FWD_FLOP * 51 / (res["network_forward_ms_51_maps"] * 1e-3) / 1e12,
                     "peak": PEAKS.get("bf16_tflops"), "unit": "TFLOP/s",
                     "frac": (NET_FWD_FLOP * 51 / (res["network_forward_ms_51_maps"] * 1e-3) / 1e12
                              / PEAKS["bf16_tflops"]) if "bf16_tflops" in PEAKS else None,
                     "peak_source": "measured cuBLAS bf16 (burst)", "traffic": None},
        "gpu_launches": None, "clocks": sampler.summary()}
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    ctx.close()


# ---------------------------------------------------------------------------------------------
# Follow-up of candidates (Sec. V)
# ---------------------------------------------------------------------------------------------

FOLLOWUP_T_FFT = 8.0        # twice the search's T_FFT


def followup_candidates(spec):
    """One candidate per injection of the series, off the truth by 0.3 of a search bin in f0 and by
    one fdot step of the follow-up grid (df / T_obs) in spin-down."""
    from paper_1810_09784_gb300 import synth
    out = []
    for inj in spec.injections:
        dfdot = (1.0 / FOLLOWUP_T_FFT) / spec.t_obs
        k = inj.k + dfdot / inj.f0 ** inj.n
        out.append(synth.Injection(f0=inj.f0 + 0.3 * spec.df, k=k, n=inj.n, amp=inj.amp))
    return out


def followup_oracle(spec, x, cand):
    """The oracle's follow-up of one candidate: heterodyne, complex peakmap, n = 0 Hough map,
    candidate, projection.  Returns (seconds, peaks)."""
    from oracle import gfh_oracle as O
    (lo, hi), f = workloads.followup_fields(cand, spec.t_obs, FOLLOWUP_T_FFT)
    t0 = time.perf_counter()
    z = O.heterodyne(x, spec.fs, 0.0, cand.f0, cand.k, cand.n).astype(np.complex64)
    fi, bj = O.peakmap_complex(z, spec.fs, FOLLOWUP_T_FFT, lo, hi)
    og = O.make_grid(O.Grid(**{k: v for k, v in f.items() if k != "list"}))
    hm = O.hough_map(og, fi, bj)
    best = max(O.select_candidates(og, hm)[0], key=lambda c: c["count"])
    O.project_peaks(fi, bj, f["t_first"], f["t_hop"], f["df"], best["fdot0"], lo, hi)
    return time.perf_counter() - t0, len(fi)


def reference_followup(args):
    spec, _, _ = workloads.plain_paper(seed=2)
    x = spec.series()
    cands = followup_candidates(spec)
    vals = []
    for i in range(args.warmup + args.steps):
        sec, _ = followup_oracle(spec, x, cands[i % len(cands)])
        if i >= args.warmup:
            vals.append(sec)
    value = 1.0 / float(np.mean(vals))
    sample = ("oracle follow-up of one candidate per step (numpy heterodyne of the 41.3M-sample "
              "series, complex FFTs, n = 0 Hough map, projection), 1 thread")
    print(json.dumps({"impl": "reference", "metric": "candidate follow-ups/s", "value": value,
                      "unit": "candidates/s", "n_gpus": args.gpus, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(vals)),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                      "dtype": "fp64 phase, complex64 series, int32 counts", "data": "synthetic",
                      "config": {"workload": "followup (one candidate per step on the CPU)"},
                      "cpu_baseline": {"value": value, "unit": "candidates/s", "cores": 1,
                                       "kind": "oracle", "sample": sample},
                      "e2e": {"value": value, "unit": "candidates/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def run_followup(args):
    """Sec. V follow-up of the 20 injections of the 10080 s, 4096 Hz series: for each candidate the
    peakmap of the series corrected by it (8 s frames, f0 +- 5 Hz; the one-pass heterodyne + band
    spectra + peak search), the original FrequencyHough (n = 0, 32 fdot rows) with its candidate,
    and the projection with the residual spin-down.  One step = all 20 candidates.  The two-call
    form (heterodyne of the whole series, then 32768-point complex FFTs) is timed beside it."""
    import torch

    from paper_1810_09784_gb300 import build as _build
    from paper_1810_09784_gb300 import gfh

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    stream = torch.cuda.Stream()
    ctx = gfh.Context(local, stream)
    spec, _, _ = workloads.plain_paper(seed=ranks.rank_seed(2, rank))
    series_np = spec.series()
    x_host = torch.from_numpy(series_np).pin_memory()
    x_dev = x_host.cuda()
    z = torch.empty(2 * series_np.size, dtype=torch.float32, device="cuda")
    cands = followup_candidates(spec)
    setups = []
    for c in cands:
        (lo, hi), f = workloads.followup_fields(c, spec.t_obs, FOLLOWUP_T_FFT)
        g = gfh.grid_make(gfh.Grid(**f))
        hmap = torch.empty((g.n_k, g.ld_x0), dtype=torch.int32, device="cuda")
        cd = torch.empty(g.n_bands * gfh.CANDIDATE_BYTES, dtype=torch.uint8, device="cuda")
        plan = gfh.Plan(ctx, [g], [hmap], [cd], None)
        counts = torch.empty(hi - lo + 1, dtype=torch.int32, device="cuda")
        setups.append((c, lo, hi, f, g, plan, cd, counts))
    n_fft2 = (series_np.size - int(spec.fs * FOLLOWUP_T_FFT)) // int(spec.fs * FOLLOWUP_T_FFT / 2) + 1
    cap = n_fft2 * 100
    fo = torch.empty(cap, dtype=torch.int32, device="cuda")
    bo = torch.empty(cap, dtype=torch.int32, device="cuda")
    off = torch.zeros(2, dtype=torch.int64, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)
    results = []

    def step(h2d=False, het_events=None, out=None, two_call=False):
        if h2d:
            x_dev.copy_(x_host, non_blocking=True)
        for q, (c, lo, hi, f, g, plan, cd, counts) in enumerate(setups):
            if het_events is not None:
                het_events[q][0].record(stream)
            if two_call:
                ctx.heterodyne(x_dev, spec.fs, 0.0, c.f0, c.k, c.n, z)
                if het_events is not None:
                    het_events[q][1].record(stream)
                n = ctx.peakmap_complex(z, spec.fs, FOLLOWUP_T_FFT, lo, hi, 2.5, fo, bo)
            else:
                n = ctx.heterodyne_band_peaks(x_dev, spec.fs, 0.0, c.f0, c.k, c.n, FOLLOWUP_T_FFT,
                                              lo, hi, 2.5, fo, bo)
                if het_events is not None:
                    het_events[q][1].record(stream)
            off[1] = n
            plan.execute(fo, bo, off, 1)
            rec = gfh.candidates_to_numpy(cd)
            best = rec[np.argmax(rec["count"])]
            ctx.project_peaks(fo, bo, n, f["t_first"], f["t_hop"], f["df"], float(best["fdot0"]),
                              lo, hi, counts)
            if out is not None:
                cnt = counts.cpu().numpy()
                out.append((int(best["count"]), float(best["cr"]), float(best["f0"]), c,
                            float(cnt.max()), n))

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        step(out=results)
        torch.cuda.synchronize()
        if ctx.check() != gfh.GFH_OK:
            raise RuntimeError("input check failed")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    with sampler, torch.cuda.stream(stream):
        barrier()
        a, b = ev(), ev()
        het = [[(ev(), ev()) for _ in setups] for _ in range(args.steps)]
        a.record(stream)
        for i in range(args.steps):
            step(het_events=het[i])
        b.record(stream)
        barrier()
        ms = a.elapsed_time(b) / args.steps
    clocks = sampler.summary()
    ms_band = sum(e0.elapsed_time(e1) for st in het for e0, e1 in st) / (args.steps * len(setups))
    ms_max, total = ranks.combine(ms, float(len(setups)), device="cuda")
    value = total / (ms_max * 1e-3)
    # the two-call form on the same candidates: heterodyne of the series, then full complex FFTs
    with torch.cuda.stream(stream):
        step(two_call=True)
        barrier()
        het2 = [[(ev(), ev()) for _ in setups] for _ in range(args.steps)]
        a.record(stream)
        for i in range(args.steps):
            step(het_events=het2[i], two_call=True)
        b.record(stream)
        barrier()
        ms_two = a.elapsed_time(b) / args.steps
    ms_het = sum(e0.elapsed_time(e1) for st in het2 for e0, e1 in st) / (args.steps * len(setups))
    with torch.cuda.stream(stream):
        barrier()
        a.record(stream)
        for _ in range(args.steps):
            step(h2d=True)
            for s_ in setups:
                s_[7].cpu()
        b.record(stream)
        barrier()
        ms_e2e = ranks.combine(a.elapsed_time(b) / args.steps, 0.0, device="cuda")[0]
    if rank != 0:
        ctx.close()
        return
    het_bytes = series_np.size * 12
    achieved_het = het_bytes / (ms_het * 1e-3) / 1e9
    # band spectra: P = N / J column transforms of J points (J/2 log2 J radix-2 butterflies of 10
    # flops) and the twiddled sum over the P residues (P J complex multiply-adds of 8 flops)
    N = int(round(spec.fs * FOLLOWUP_T_FFT))
    J = 256
    P = N // J
    flops_frame = P * (J // 2) * int(math.log2(J)) * 10 + P * J * 8
    frames = (series_np.size - N) // (N // 2) + 1
    achieved = flops_frame * frames / (ms_band * 1e-3) / 1e12
    fp32_peak = ctx.sms() * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    recovered = sum(1 for r in results if abs(r[2] - r[3].f0 + 0.3 * spec.df) < 1.0 and r[1] > 5.0)
    line = {
        "metric": "candidate follow-ups/s", "value": value, "unit": "candidates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp64 anchors + 64-bit fixed-point phase, complex64 series, int32 counts",
        "data": "synthetic",
        "config": {"workload": "followup: the 20 injections of the 10080 s, 4096 Hz series, each from a "
                               "candidate 0.3 bin and one fdot step off; heterodyne, 8 s complex FFTs, "
                               "peakmap in f0 +- 5 Hz, original FrequencyHough (n = 0, 32 fdot rows), "
                               "projection",
                   "candidates": len(setups), "samples": int(series_np.size),
                   "l2": "series 165 MB read per candidate (larger than L2)",
                   "timing": "direct calls (two host reads per candidate: peak count, top candidate)"},
        "breakdown_ms": {"step": ms, "band_peaks_per_candidate": ms_band,
                         "rest_per_candidate": ms / len(setups) - ms_band},
        "two_call_form": {"ms_per_step": ms_two, "heterodyne_ms_per_candidate": ms_het,
                          "speedup_one_pass": ms_two / ms,
                          "heterodyne_roofline": {"bound": "hbm", "achieved": achieved_het,
                                                  "peak": HBM_PEAK, "unit": "GB/s",
                                                  "frac": achieved_het / HBM_PEAK,
                                                  "algorithmic": "12 bytes per sample"}},
        "roofline": {"bound": "alu", "kernel": "k_band_dft", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "peak_source": "derived: device SM count x 128 fp32 FMA/clk x 2 flops x max SM clock",
                     "algorithmic": f"{flops_frame} flops per {N}-sample frame ({J} bins), {frames} frames; "
                                    "the timed call also holds the anchor pass and the band peak search",
                     "traffic": None},
        "followup": {"recovered": recovered, "of": len(results),
                     "fh_count_cr_f0": [[r[0], round(r[1], 2), round(r[2], 4)] for r in results]},
        "e2e": {"value": total / (ms_e2e * 1e-3), "unit": "candidates/s",
                "h2d_bytes_per_step": series_np.size * 4,
                "d2h_bytes_per_step": sum(s_[7].numel() * 4 + s_[6].numel() for s_ in setups),
                "ms_per_step": ms_e2e},
        "gpu_launches": 11 * len(setups) * args.steps,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        sec, _ = followup_oracle(spec, series_np, cands[0])
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": "candidates/s", "cores": 1,
                                "kind": "oracle",
                                "sample": "oracle follow-up of the first candidate (full series), 1 thread"}
    print(json.dumps(line), flush=True)
    for s_ in setups:
        s_[5].close()
    ctx.close()


# ---------------------------------------------------------------------------------------------
# Longer FFTs for later times (Sec. VI.D)
# ---------------------------------------------------------------------------------------------

def splice_setup(spec):
    """The plain_paper series split by the Sec. VI.D planner for the family n = 5, f0 <= 2000 Hz,
    |fdot0| <= 1/(2 s)^2, starting from 2 s FFTs (three levels): each portion searched in the 19
    sub-band maps of plain_paper above 100 Hz (100 Hz analysis bands + 50 Hz extension, 2000 k
    rows)."""
    from paper_1810_09784_gb300 import gfh, splice
    portions = gfh.tfft_portions(5.0, 2000.0, 0.25, 2.0, spec.t_obs, 3)
    bands = []
    a = 100.0             # the equaliser's 128-bin warm-up needs bin_lo >= 130 at 2 s FFTs
    while a < 2000.0 - 1e-9:
        bands.append((a, min(a + 100.0, 2000.0)))
        a += 100.0
    plan = splice.portion_plan(portions, spec.fs, spec.n_samples, 5.0, bands, 2000, ext=50.0)
    for P in plan:        # the extension stops at the band's top, as in plain_paper
        for f in P.fields:
            f["bin_hi"] = min(f["bin_hi"], int(round(2000.0 * P.t_fft)) - 1)
    return plan


def reference_splice(args):
    from oracle import gfh_oracle as O
    spec, _, _ = workloads.plain_paper(seed=2)
    x = spec.series()
    plan = splice_setup(spec)
    vals, times = [], []
    for i in range(args.warmup + args.steps):
        t_step, updates = 0.0, 0
        for P in plan:
            lo = min(f["bin_lo"] for f in P.fields)
            hi = max(f["bin_hi"] for f in P.fields)
            t0 = time.perf_counter()
            fi, bj = O.peakmap(x[P.s_begin:P.s_end], spec.fs, P.t_fft, lo, hi)
            t_step += time.perf_counter() - t0
            for f in P.fields:
                og = O.make_grid(O.Grid(**{k: v for k, v in f.items() if k != "list"}))
                sel = (bj >= og.bin_lo) & (bj <= og.bin_hi)
                updates += int(sel.sum()) * og.n_k
                t1 = time.perf_counter()
                O.hough_row(og, fi, bj, og.n_k // 2)
                t_step += (time.perf_counter() - t1) * og.n_k
        if i >= args.warmup:
            vals.append(updates / t_step)
            times.append(t_step)
    value = float(np.mean(vals))
    sample = ("oracle peakmaps of every portion + one k row of each map, extrapolated to all rows; "
              "numpy, 1 thread")
    print(json.dumps({"impl": "reference", "metric": "Hough updates/s (peaks x k-bins)",
                      "value": value, "unit": "updates/s", "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None,
                      "dtype": "int32 counts, fp32 spectra, fp64 grid", "data": "synthetic",
                      "config": {"workload": "splice (CPU oracle)"},
                      "cpu_baseline": {"value": value, "unit": "updates/s", "cores": 1,
                                       "kind": "oracle", "sample": sample},
                      "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def run_splice(args):
    """Sec. VI.D on the plain_paper series: one step = every portion's peakmap (its own FFT length,
    on its samples) and its 20 sub-band maps with candidates, then the coincidences of each
    sub-band's candidates between consecutive portions."""
    import torch

    from paper_1810_09784_gb300 import build as _build
    from paper_1810_09784_gb300 import gfh, splice

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    stream = torch.cuda.Stream()
    ctx = gfh.Context(local, stream)
    spec, _, _ = workloads.plain_paper(seed=ranks.rank_seed(2, rank))
    series_np = spec.series()
    x_host = torch.from_numpy(series_np).pin_memory()
    x_dev = x_host.cuda()
    plan = splice_setup(spec)
    parts = []
    for P in plan:
        grids = [gfh.grid_make(gfh.Grid(**f)) for f in P.fields]
        maps = [torch.empty((g.n_k, g.ld_x0), dtype=torch.int32, device="cuda") for g in grids]
        cands = [torch.empty(g.n_bands * gfh.CANDIDATE_BYTES, dtype=torch.uint8, device="cuda")
                 for g in grids]
        hp = gfh.Plan(ctx, grids, maps, cands, None, tile=(16, 3072, 1024))
        lo = min(f["bin_lo"] for f in P.fields)
        hi = max(f["bin_hi"] for f in P.fields)
        n_fft = P.fields[0]["n_fft"]
        cap = int(n_fft * (hi - lo + 1) * 0.12) + 1024
        fo = torch.empty(cap, dtype=torch.int32, device="cuda")
        bo = torch.empty(cap, dtype=torch.int32, device="cuda")
        off = torch.zeros(2, dtype=torch.int64, device="cuda")
        parts.append(dict(P=P, grids=grids, maps=maps, cands=cands, plan=hp, lo=lo, hi=hi, fo=fo,
                          bo=bo, off=off))
    n_bands_total = [sum(g.n_bands for g in p["grids"]) for p in parts]
    match = torch.empty(max(n_bands_total), dtype=torch.int32, device="cuda")
    dist_t = torch.empty(max(n_bands_total), dtype=torch.float64, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(h2d=False, hough_events=None, src=None):
        if h2d and src is None:                  # the series copied on this stream
            x_dev.copy_(x_host, non_blocking=True)
        src = x_dev if src is None else src
        for q, p in enumerate(parts):
            P = p["P"]
            ctx.peakmap_async(src[P.s_begin:P.s_end], spec.fs, P.t_fft, p["lo"], p["hi"],
                              2.5, p["fo"], p["bo"], p["off"][1:2])
            if hough_events is not None:
                hough_events[q][0].record(stream)
            p["plan"].execute(p["fo"], p["bo"], p["off"], 1)
            if hough_events is not None:
                hough_events[q][1].record(stream)
        for pa, pb in zip(parts, parts[1:]):
            for ga, ca, gb, cb in zip(pa["grids"], pa["cands"], pb["grids"], pb["cands"]):
                ctx.coincide(ca, ga.n_bands, cb, gb.n_bands, max(ga.dx0, gb.dx0),
                             max(ga.dk, gb.dk), 3.0, match, dist_t)
        if h2d:
            for p, hc in zip(parts, cand_host):
                for c, h in zip(p["cands"], hc):
                    h.copy_(c, non_blocking=True)

    cand_host = [[torch.empty_like(c, device="cpu").pin_memory() for c in p["cands"]] for p in parts]
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if ctx.check() != gfh.GFH_OK:
            raise RuntimeError("input check failed")
    updates = 0
    for p in parts:
        n = int(p["off"][1].item())
        updates += splice.update_count(p["grids"], p["bo"][:n].cpu().numpy())

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    with sampler, torch.cuda.stream(stream):
        barrier()
        a, b = ev(), ev()
        hev = [[(ev(), ev()) for _ in parts] for _ in range(args.steps)]
        torch.cuda.nvtx.range_push("timed_steps")
        a.record(stream)
        for i in range(args.steps):
            step(hough_events=hev[i])
        b.record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
        ms = a.elapsed_time(b) / args.steps
    clocks = sampler.summary()
    ms_hough = sum(e0.elapsed_time(e1) for st in hev for e0, e1 in st) / args.steps
    ms_max, total = ranks.combine(ms, float(updates), device="cuda")
    value = total / (ms_max * 1e-3)
    # end to end: each step's series copied from pinned host memory on a copy stream into one of
    # two device buffers (overlapping the previous step's search), its candidates read back
    x_buf = [x_dev, torch.empty_like(x_dev)]
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]
    h2d_ev = [(ev(), ev()) for _ in range(args.steps)]

    def e2e_step(i, timed=False):
        k = i & 1
        copy_stream.wait_event(consumed[k])              # buffer k no longer read
        if timed:
            h2d_ev[i][0].record(copy_stream)
        with torch.cuda.stream(copy_stream):
            x_buf[k].copy_(x_host, non_blocking=True)
        copied[k].record(copy_stream)
        if timed:
            h2d_ev[i][1].record(copy_stream)
        stream.wait_event(copied[k])
        with torch.cuda.stream(stream):
            step(h2d=True, src=x_buf[k])
        consumed[k].record(stream)

    for i in range(max(args.warmup, 2)):                # untimed: both buffers used once
        e2e_step(i)
    barrier()
    a.record(stream)
    copy_stream.wait_event(a)
    for i in range(args.steps):
        e2e_step(i, timed=True)
    b.record(stream)
    barrier()
    ms_e2e = ranks.combine(a.elapsed_time(b) / args.steps, 0.0, device="cuda")[0]
    ms_h2d = sum(e0.elapsed_time(e1) for e0, e1 in h2d_ev) / args.steps
    # coincidences of the injections between the two portions (top candidate of each band)
    coinc = None
    if len(parts) >= 2:
        pa, pb = parts[0], parts[1]
        hits, tot = 0, 0
        for ga, ca, gb, cb in zip(pa["grids"], pa["cands"], pb["grids"], pb["cands"]):
            m_, d_ = splice.coincide(ctx, ca, ga, cb, gb)
            torch.cuda.synchronize()              # the kernel ran on the library's stream
            ra = gfh.candidates_to_numpy(ca)
            m_ = m_.cpu().numpy()
            strong = ra["cr"] > 6.0
            tot += int(strong.sum())
            hits += int((strong & (m_ >= 0)).sum())
        coinc = {"strong_candidates_first_portion": tot, "with_a_coincidence_in_the_second": hits}
    if rank != 0:
        ctx.close()
        return
    atomics = 2.0 * updates
    achieved = atomics / (ms_hough * 1e-3) / 1e9
    line = {
        "metric": "Hough updates/s (peaks x k-bins)", "value": value, "unit": "updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32 counts, fp32 spectra, fp64 grid", "data": "synthetic",
        "config": {"workload": "splice: the plain_paper series in Sec. VI.D portions (n = 5, f0 <= 2000 Hz, "
                               "|fdot0| <= 0.25 Hz/s, T_FFT 2 s then 4 s), 19 sub-band maps (100-2000 Hz) "
                               "of 2000 k rows per portion, coincidences between the portions",
                   "portions": [[p["P"].t_fft, p["P"].s_begin / spec.fs, p["P"].s_end / spec.fs]
                                for p in parts],
                   "maps": sum(len(p["grids"]) for p in parts), "updates_per_step": updates,
                   "tile": [16, 3072, 1024],
                   "l2": "inputs larger than L2 (series 165 MB, maps %d MB per step)"
                         % (sum(g.n_k * g.ld_x0 * 4 for p in parts for g in p["grids"]) // 1000000),
                   "timing": "direct calls"},
        "breakdown_ms": {"step": ms, "hough_select": ms_hough, "rest": ms - ms_hough},
        "roofline": {**atomic_roofline(ctx, stream, achieved), "traffic": None},
        "coincidences": coinc,
        "e2e": {"value": total / (ms_e2e * 1e-3), "unit": "updates/s",
                "h2d_bytes_per_step": series_np.size * 4,
                "d2h_bytes_per_step": sum(c.numel() for p in parts for c in p["cands"]),
                "ms_per_step": ms_e2e, "h2d_ms_per_copy": ms_h2d,
                "h2d_gbs": series_np.size * 4 / (ms_h2d * 1e-3) / 1e9,
                "timing": "asynchronous public calls after untimed warm-up steps; each step's "
                          "series copied from pinned host memory on a copy stream into one of two "
                          "device buffers (overlapping the previous step's search) and its "
                          "candidates read back"},
        "gpu_launches": (len(parts) * 9 + len(parts[0]["grids"]) * (len(parts) - 1)) * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    for p in parts:
        p["plan"].close()
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven":
        run_gpu_lists(args)
    elif args.workload == "proposer":
        run_proposer(args)
    elif args.workload == "followup":
        run_followup(args)
    elif args.workload == "splice":
        run_splice(args)
    elif args.workload == "train":
        run_train(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
