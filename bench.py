"""Benchmark of the correction engine (one JSON line on rank 0).

Metric: Gvertices/s to zero-mismatch correction of a 512^3 Perlin field
prequantized with relative error bound 1e-4 (5 octaves, period 64, seed 2):
the vertices of the field divided by the device time from f and fhat resident
in HBM to the corrected field and the sorted edit list complete.  One step =
one msz_correct call (the whole hot path: codes, every sweep, edit list).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU, each rank correcting its own
512^3 field (independent problems: weak scaling, no collective on the data
path); value = all ranks' vertices / the slowest rank's time.
--impl reference times the CPU oracle (single thread, as it stands) on a
bounded z-slab of the same field.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

SHAPE = (512, 512, 512)  # (nz, ny, nx); --shape overrides (profiling captures only)
SEED = 2
EB_REL = 1e-4
METRIC = "Gvertices/s to zero-mismatch correction at 512\u00b3 (plain vs learned); HBM GB/s"
UNIT = "Gvertices/s"
def workload_name():
    nz, ny, nx = SHAPE
    return f"perlin3d_prequant_{nx}x{ny}x{nz}"


def workload_config(n):
    return {"workload": workload_name(), "field": "fractal Perlin noise, 5 octaves, base period 64, min-max scaled to [0,1]",
            "fhat": "2*xi*round(f/(2*xi)) (uniform prequantization)", "eb_rel": EB_REL, "seed": SEED,
            "n_vertices": n, "neighbourhood": "Freudenthal, 14 neighbours", "rule": "halve",
            "l2": "no flush: inputs f+fhat (1.07 GB) exceed the 129 MB L2"}


def load_bf16_peak():
    """Dense BF16 tensor peak: the measured cuBLAS burst figure (a conv layer is
    timed on its own), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured (burst)"
    except Exception:
        return 1900.0, "fallback"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms; only the
    samples read between mark_start() and mark_end() (the timed region) count."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_end(self):
        self.t1 = time.perf_counter()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ts, ln in self.lines:
            if self.t0 is not None and not (self.t0 <= ts <= (self.t1 or ts) + 0.06):
                continue
            parts = [p.strip() for p in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- roofline
def algorithmic_bytes(n: int, log: np.ndarray, edited: int, uncertified: int) -> int:
    """Compulsory HBM bytes of one correction:
    sweep 0 reads f, fhat and writes g (12 B/vertex) and the code of f at
    each uncertified vertex (1 B; no other vertex's code is ever read); a later sweep
    reads g and codes_f of every examined vertex (5 B each: the whole grid for
    dense sweeps, the worklist otherwise); every distinct target reads f and g
    and writes g (12 B); the edit list reads the edited bitmap (N/8 B) and
    writes 8 B per edit."""
    total = 12 * n + uncertified
    for k in range(1, log.shape[0]):
        total += 5 * int(log[k, 0])
    total += 12 * int(log[:, 2].sum())
    total += n // 8 + 8 * edited
    return total


def codes_bytes(n: int, uncertified: int) -> int:
    """Compulsory HBM bytes of sweep 0's pass (k_codes): f and fhat read, g
    written (12 B/vertex), the code of f written at each uncertified vertex."""
    return 12 * n + uncertified


# ALU operations of one steepest-neighbour code over the 14 neighbours and
# the vertex itself: per candidate and direction a compare, a value select and
# a slot select (3 ops).  The certification of sweep 0 keeps only the two
# largest and two smallest values, taking the 15 values as 7 pairs of one row
# segment plus one: the first pair sets them (2 ops: the pair's max and min),
# each further pair takes 8 (its max and min; per direction a NaN-propagating
# min / max against the leader, a three-input max / min into the runner-up and
# one into the leader), the single value 4.
ALU_OPS_CODE = 14 * 2 * 3
ALU_OPS_CERT = 2 + 6 * 8 + 4


def algorithmic_alu_ops(n: int, log: np.ndarray, uncertified: int) -> int:
    """ALU operations of one correction: the certification of every vertex,
    the codes of f and g at the uncertified vertices in sweep 0, and the codes
    of g at every vertex examined by a later sweep (dense sweeps examine the
    uncertified ones)."""
    total = ALU_OPS_CERT * n + 2 * ALU_OPS_CODE * uncertified
    for k in range(1, log.shape[0]):
        total += ALU_OPS_CODE * min(int(log[k, 0]), uncertified)
    return total


def codes_alu_ops(n: int, uncertified: int) -> int:
    """ALU operations of sweep 0's pass: the certification of every vertex
    and the codes of f and g at the uncertified ones."""
    return ALU_OPS_CERT * n + 2 * ALU_OPS_CODE * uncertified


def alu_peak(sm_mhz: float) -> float:
    """ALU-pipe peak of a GB300 in operations/s: 152 SMs x 4 sub-partitions x
    16 lanes (a warp instruction every 2 cycles) x the SM clock."""
    return 152 * 4 * 16 * sm_mhz * 1e6


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- ours
def run_ours(args, ws, rank, local):
    import torch

    from paper_2601_01787_gb300 import api, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fl = synth.perlin3d_prequant(SHAPE, seed=SEED, eb_rel=EB_REL)
    n = fl.n
    f = torch.from_numpy(fl.f).to(dev)
    fh = torch.from_numpy(fl.fhat).to(dev)
    out = torch.empty_like(f)
    cap = n // 4
    eidx = torch.empty(cap, dtype=torch.int32, device=dev)
    edel = torch.empty(cap, dtype=torch.float32, device=dev)
    ws_buf = api.workspace(api.workspace_size(f.shape), dev)
    stream = torch.cuda.current_stream(dev)

    def step(log=0, events=None):
        return api.correct(f, fh, fl.xi, out=out, edit_idx=eidx, edit_delta=edel, edit_capacity=cap,
                           ws=ws_buf, stream=stream, log_capacity=log, events=events)

    clocks = ClockSampler(local)
    clocks.start()
    first = step(log=4096)
    assert first.status == api.OK, api.status_str(first.status)
    for _ in range(max(args.warmup - 1, 0)):
        step()
    time.sleep(0.2)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # per step: before sweep 0's kernel (k_codes), between it and the loop
    # kernel (k_correct), after the loop kernel -- recorded by the library on
    # the launching stream; created here (first record) outside the timed region
    kev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(args.steps)]
    for e in [x for t in ev + kev for x in t]:
        e.record(stream)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.mark_start()
    t_wall = time.perf_counter()
    kernel_ns = []
    for i in range(args.steps):
        ev[i][0].record(stream)
        r = step()
        ev[i][1].record(stream)
        kernel_ns.append(r.stats["kernel_ns"])
        assert r.status == api.OK
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - t_wall
    # the same steps again with the library recording events around each
    # kernel (instrumentation kept out of the timed steps above)
    for i in range(args.steps):
        r = step(events=kev[i])
        assert r.status == api.OK
    torch.cuda.synchronize()
    clocks.mark_end()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_local = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms_local, ws)
    value = ws * n / (ms * 1e-3) / 1e9

    # rooflines of the two correction kernels, each over its own CUDA-event
    # launch time: k_codes (sweep 0's pass, the dominant one) and k_correct
    # (the later sweeps and the edit list)
    peak, peak_kind = load_peaks()
    log = first.sweep_log
    unc = first.stats["uncertified"]
    alg = algorithmic_bytes(n, log, first.edit_count, unc)
    alg_codes = codes_bytes(n, unc)
    alg_loop = alg - alg_codes
    kernel_ms = statistics.mean(kernel_ns) / 1e6
    codes_ms = statistics.mean(a.elapsed_time(b) for a, b, _ in kev)
    loop_ms = statistics.mean(b.elapsed_time(c) for _, b, c in kev)
    codes_gbs = alg_codes / (codes_ms * 1e-3) / 1e9
    loop_gbs = alg_loop / (loop_ms * 1e-3) / 1e9
    # the records were taken of the 512^3 workload: none for a --shape run
    full = SHAPE == (512, 512, 512)
    traffic_codes = traffic_record("k_codes_perlin512_traffic.json", "msz_correct.cu") if full else None
    traffic_loop = traffic_record("k_correct_perlin512_traffic.json", "msz_correct.cu") if full else None

    # k_codes against the ALU-pipe peak (the pipe that bounds it)
    alu_ops = codes_alu_ops(n, unc)
    alu_pk = alu_peak(clk.get("sm_mhz") or 2070.0) / 1e9
    alu_ach = alu_ops / (codes_ms * 1e-3) / 1e9

    # verification of the result (codes, labels by pointer jumping, counts)
    # and the SNAP edit rule on the same field
    def timed_ms(fn, reps=3):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            res = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, res

    verify_ms, ver = timed_ms(lambda: api.verify(f, out))
    snap_ms, snap = timed_ms(lambda: api.correct(f, fh, fl.xi, rule="snap", out=out, edit_idx=eidx, edit_delta=edel,
                                                 edit_capacity=cap, ws=ws_buf, stream=stream))
    ws_below = api.workspace(api.load().msz_workspace_size_rule(api.grid_of(f.shape), 2), dev)
    below_ms, below = timed_ms(lambda: api.correct(f, fh, fl.xi, rule="below", out=out, edit_idx=eidx,
                                                   edit_delta=edel, edit_capacity=cap, ws=ws_below, stream=stream))
    step()  # leave the HALVE result in out
    stream_stats = edit_stream(fh, out, eidx, first.edit_count, stream)

    # end to end through the host-buffer entry point (pinned buffers)
    hf = torch.from_numpy(fl.f).pin_memory()
    hfh = torch.from_numpy(fl.fhat).pin_memory()
    hout = torch.empty(fl.shape, dtype=torch.float32).pin_memory()
    hidx = torch.empty(cap, dtype=torch.int32).pin_memory()
    hdel = torch.empty(cap, dtype=torch.float32).pin_memory()
    hws = api.workspace(api.host_workspace_size(fl.shape, cap), dev)
    e2e_steps = max(10, args.steps // 2)

    def hstep():
        return api.correct_host(hf, hfh, fl.xi, out=hout, edit_idx=hidx, edit_delta=hdel, edit_capacity=cap,
                                ws=hws, stream=stream)

    for _ in range(2):
        hr = hstep()
    assert hr.status == api.OK
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        hr = hstep()
    torch.cuda.synchronize()
    serial_ms = max_over_ranks((time.perf_counter() - t0) / e2e_steps * 1e3, ws)

    # end to end through the pipelined host-buffer entry points: the same
    # copies every step, consecutive steps overlapped (two result buffers)
    del hws
    api._ws_cache.clear()
    pl = api.Pipeline(fl.shape, edit_capacity=cap, device=dev)
    hout2 = torch.empty(fl.shape, dtype=torch.float32).pin_memory()
    hidx2 = torch.empty(cap, dtype=torch.int32).pin_memory()
    hdel2 = torch.empty(cap, dtype=torch.float32).pin_memory()
    sets = [(hout, hidx, hdel), (hout2, hidx2, hdel2)]

    def run_pipeline(steps):
        last = None
        for i in range(steps):
            if i >= 2:
                last = pl.collect()
                assert last.status == api.OK, api.status_str(last.status)
            pl.submit(hf, hfh, fl.xi, *sets[i % 2])
        for _ in range(min(steps, 2)):
            last = pl.collect()
            assert last.status == api.OK, api.status_str(last.status)
        return last

    run_pipeline(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hr = run_pipeline(e2e_steps)
    torch.cuda.synchronize()
    field_ms = max_over_ranks((time.perf_counter() - t0) / e2e_steps * 1e3, ws)
    assert hr.edit_count == first.edit_count
    pl.close()
    del pl

    # ... and through the encoded pipeline: each step's result is the edit
    # list's stream (what a compressor stores beside its data), encoded on
    # the device, instead of g
    ple = api.Pipeline(fl.shape, edit_capacity=cap, device=dev, encoded=True)
    sbufs = [torch.empty(ple.stream_bound(), dtype=torch.uint8).pin_memory() for _ in range(2)]

    def run_encoded(steps):
        last = None
        for i in range(steps):
            if i >= 2:
                last = ple.collect()
                assert last.status == api.OK, api.status_str(last.status)
            ple.submit(hf, hfh, fl.xi, sbufs[i % 2])
        for _ in range(min(steps, 2)):
            last = ple.collect()
            assert last.status == api.OK, api.status_str(last.status)
        return last

    run_encoded(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    he = run_encoded(e2e_steps)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) / e2e_steps * 1e3, ws)
    e2e_value = ws * n / (e2e_ms * 1e-3) / 1e9
    assert he.edit_count == first.edit_count
    stream_len = int(he.stream.numel())
    ple.close()
    del ple, sbufs
    link = link_reference(hf, hfh, f, fh, stream)

    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(n) | {"parallelism": f"independent fields x{ws}" if ws > 1 else "single"},
        # the dominant kernel (sweep 0's pass) against the measured HBM copy
        # peak: its algorithmic bytes over its CUDA-event launch time
        "roofline": {"bound": "hbm", "achieved": round(codes_gbs, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(codes_gbs / peak, 4), "traffic": traffic_codes, "peak_kind": peak_kind,
                     "algorithmic_bytes": alg_codes, "kernel": "k_codes<TMA>", "kernel_ms": round(codes_ms, 5),
                     "share_of_step": round(codes_ms / ms_local, 4)},
        # the other kernel: the later sweeps and the edit list
        "roofline_loop": {"bound": "hbm", "achieved": round(loop_gbs, 2), "peak": peak, "unit": "GB/s",
                          "frac": round(loop_gbs / peak, 4), "traffic": traffic_loop, "peak_kind": peak_kind,
                          "algorithmic_bytes": alg_loop, "kernel": "k_correct<3, TMA>",
                          "kernel_ms": round(loop_ms, 5), "share_of_step": round(loop_ms / ms_local, 4)},
        # the whole correction: algorithmic bytes over the step time, and over
        # the device time from sweep 0's start to the end of the loop kernel
        "roofline_step": {"achieved": round(alg / (ms_local * 1e-3) / 1e9, 2), "unit": "GB/s",
                          "frac": round(alg / (ms_local * 1e-3) / 1e9 / peak, 4), "algorithmic_bytes": alg,
                          "kernel_ms_device": round(kernel_ms, 5),
                          "frac_kernel_time": round(alg / (kernel_ms * 1e-3) / 1e9 / peak, 4)},
        # a model, not a measurement: modelled ALU operations of k_codes over
        # a peak derived from the unit counts and the sampled clock
        "roofline_alu_model": {"bound": "alu", "kernel": "k_codes<TMA>", "achieved": round(alu_ach, 1),
                               "peak": round(alu_pk, 1), "unit": "Gop/s", "frac": round(alu_ach / alu_pk, 4),
                               "ops": alu_ops, "uncertified": unc,
                               "peak_kind": "derived: 152 SMs x 64 ALU lanes x median SM clock"},
        "verify": {"ms": round(verify_ms, 4), "codes_equal": ver["codes_equal"], "wrong_labels": ver["wrong_labels"],
                   "false_extrema": ver["fp_max"] + ver["fn_max"] + ver["fp_min"] + ver["fn_min"]},
        "rules": {"halve": {"ms": round(ms, 4), "sweeps": first.stats["sweeps"], "edits": first.stats["edits"],
                            "edited": first.edit_count},
                  "snap": {"ms": round(snap_ms, 4), "sweeps": snap.stats["sweeps"], "edits": snap.stats["edits"],
                           "edited": snap.edit_count, "status": api.status_str(snap.status)},
                  "below_reference": {"ms": round(below_ms, 4), "sweeps": below.stats["sweeps"],
                                      "edits": below.stats["edits"], "edited": below.edit_count,
                                      "status": api.status_str(below.status)}},
        "e2e": {"value": round(e2e_value, 4), "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": stream_len, "ms_per_step": round(e2e_ms, 4),
                "link": link,
                "frac_of_link": round(8 * n / (e2e_ms * 1e-3) / 1e9 / link["h2d_gbs"], 4),
                "api": "msz_pipeline_submit_encoded / msz_pipeline_collect_encoded (consecutive steps "
                       "overlapped; result: the edit list's stream)",
                "field": {"api": "msz_pipeline_submit / msz_pipeline_collect (result: g and the edit list)",
                          "ms_per_step": round(field_ms, 4), "value": round(ws * n / (field_ms * 1e-3) / 1e9, 4),
                          "d2h_bytes_per_step": 4 * n + 8 * hr.edit_count},
                "serial": {"api": "msz_correct_host (one call at a time; result: g and the edit list)",
                           "ms_per_step": round(serial_ms, 4),
                           "value": round(ws * n / (serial_ms * 1e-3) / 1e9, 4)}},
        # two kernels a correction: k_codes (sweep 0) and k_correct (the rest)
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "sweeps": first.stats["sweeps"], "edited": first.edit_count, "first_distorted": first.stats["first_distorted"],
        "edit_ratio": round(first.edit_count / n, 6),
        "edit_stream": stream_stats,
        "sweep_log": log.tolist(),
        "phase_ms": [[round(a / 1e6, 4), round(b / 1e6, 4)] for a, b in first.timeline.tolist()],
        "wall_s_timed": round(wall, 4),
    }
    if rank == 0 and not args.no_batch:
        del f, fh, out, eidx, edel, hf, hfh, hout, hidx, hdel, hout2, hidx2, hdel2, sets
        api._ws_cache.clear()
        torch.cuda.empty_cache()
        line["batch"] = run_batch(dev, stream, sm_mhz=clk.get("sm_mhz"), count=args.batch_fields)
    if rank == 0 and args.large:
        f = fh = out = None  # drop the 512^3 buffers (if the batch leg has not already)
        api._ws_cache.clear()
        torch.cuda.empty_cache()
        line["large"] = run_large(dev, stream)
    if rank == 0 and args.configs:
        f = fh = out = None
        api._ws_cache.clear()
        torch.cuda.empty_cache()
        line["configs"] = run_configs(dev, stream)
    if rank == 0 and not args.no_relaxed:
        f = fh = out = None
        api._ws_cache.clear()
        torch.cuda.empty_cache()
        line["relaxed"] = run_relaxed(dev, stream)
    if rank == 0 and not args.no_learned:
        api._ws_cache.clear()
        torch.cuda.empty_cache()
        line["learned"] = run_learned(dev, stream)
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(fl, args.cpu_slab)
        if args.configs:
            line["cpu_baseline"]["configs"] = cpu_baseline_configs()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_relaxed(dev, stream, reps: int = 3) -> dict:
    """The relaxed synchronization of Sec. IV-B (32 x 8 x 8 tiles iterating
    locally, merged by minimum) against the synchronous loop, on the 512^3
    peak field of the learned comparison and on the 512^3 Perlin field:
    device time to a corrected field, global iterations against sweeps."""
    import torch

    from paper_2601_01787_gb300 import api, synth
    out = {}
    for name, fl in (("peaks3d_512x512x512 (5000 peaks, seed 7, eb_rel 1e-4)",
                      synth.peaks3d((512, 512, 512), seed=7, eb_rel=1e-4, npeaks=5000)),
                     (workload_name(), synth.perlin3d_prequant(SHAPE, seed=SEED, eb_rel=EB_REL))):
        f = torch.from_numpy(fl.f).to(dev)
        fh = torch.from_numpy(fl.fhat).to(dev)

        def timed(fn):
            best, res = None, None
            for _ in range(reps + 1):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                res = fn()
                b.record(stream)
                torch.cuda.synchronize()
                t = a.elapsed_time(b)
                best = t if best is None else min(best, t)
            return best, res

        tp, p = timed(lambda: api.correct(f, fh, fl.xi, edit_capacity=0, stream=stream))
        tr, r = timed(lambda: api.correct_relaxed(f, fh, fl.xi, edit_capacity=0, stream=stream))
        v = api.verify(f, r.out)
        out[name] = {"plain": {"ms": round(tp, 4), "sweeps": p.stats["sweeps"]},
                     "relaxed": {"ms": round(tr, 4), "iterations": r.stats["sweeps"],
                                 "local_sweeps": r.stats["local_sweeps"], "tile_runs": r.stats["tile_runs"],
                                 "edited": r.edit_count, "plain_edited": p.edit_count,
                                 "verified": bool(v["codes_equal"] and v["wrong_labels"] == 0)}}
        del f, fh
        torch.cuda.empty_cache()
    return {"tile": list(api.RELAXED_TILE), "fields": out}


def run_large(dev, stream, reps: int = 3) -> dict:
    """The correction of one 1024^3 prequantized Perlin field (1.07e9
    vertices, 12.9 GB of f, fhat and g plus a 1.6 GB workspace)."""
    import torch

    from paper_2601_01787_gb300 import api, synth
    fl = synth.perlin3d_prequant((1024, 1024, 1024), seed=SEED, eb_rel=EB_REL)
    f = torch.from_numpy(fl.f).to(dev)
    fh = torch.from_numpy(fl.fhat).to(dev)
    del fl.f, fl.fhat
    out = torch.empty_like(f)
    cap = f.numel() // 8
    eidx = torch.empty(cap, dtype=torch.int32, device=dev)
    edel = torch.empty(cap, dtype=torch.float32, device=dev)
    best, r = None, None
    for _ in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = api.correct(f, fh, fl.xi, out=out, edit_idx=eidx, edit_delta=edel, edit_capacity=cap, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        assert r.status == api.OK, api.status_str(r.status)
        t = a.elapsed_time(b)
        best = t if best is None else min(best, t)
    n = f.numel()
    return {"workload": "perlin3d_prequant_1024x1024x1024, seed 2, eb_rel 1e-4", "n_vertices": n, "unit": UNIT,
            "value": round(n / (best * 1e-3) / 1e9, 4), "ms": round(best, 4), "sweeps": r.stats["sweeps"],
            "edited": r.edit_count, "kernel_ms": round(r.stats["kernel_ns"] / 1e6, 4)}


def run_configs(dev, stream, reps: int = 5) -> dict:
    """The two configurations the default run does not time: the 2D 256^2
    Perlin field with noise (eb_rel 1e-3) and the 1024 x 1024 x 512 Gaussian
    peak field (20,000 peaks, eb_rel 1e-4), each corrected by msz_correct with
    inputs resident on the device (best of `reps` after one warm-up)."""
    import torch

    from paper_2601_01787_gb300 import api, synth
    out = {}
    for name, make in (("perlin2d_256x256 (seed 1, eb_rel 1e-3, fhat = f + U[-xi, xi])",
                        lambda: synth.perlin2d((256, 256), seed=1, eb_rel=1e-3)),
                       ("peaks3d_1024x1024x512 (20,000 peaks, seed 3, eb_rel 1e-4, fhat = f + U[-xi, xi])",
                        lambda: synth.peaks3d((512, 1024, 1024), seed=3, eb_rel=1e-4))):
        fl = make()
        f = torch.from_numpy(fl.f).to(dev)
        fh = torch.from_numpy(fl.fhat).to(dev)
        o = torch.empty_like(f)
        cap = f.numel() // 2
        eidx = torch.empty(cap, dtype=torch.int32, device=dev)
        edel = torch.empty(cap, dtype=torch.float32, device=dev)
        ws = api.workspace(api.workspace_size(f.shape), dev)
        best, r = None, None
        for _ in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = api.correct(f, fh, fl.xi, out=o, edit_idx=eidx, edit_delta=edel, edit_capacity=cap, ws=ws,
                            stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            assert r.status == api.OK, api.status_str(r.status)
            t = a.elapsed_time(b)
            best = t if best is None else min(best, t)
        n = f.numel()
        out[name] = {"n_vertices": n, "unit": UNIT, "value": round(n / (best * 1e-3) / 1e9, 4),
                     "ms": round(best, 4), "sweeps": r.stats["sweeps"], "edited": r.edit_count,
                     "kernel_ms": round(r.stats["kernel_ns"] / 1e6, 4)}
        del f, fh, o, eidx, edel, ws, fl
        api._ws_cache.clear()
        torch.cuda.empty_cache()
    return out


def run_batch(dev, stream, reps: int = 5, sm_mhz: float | None = None, count: int = 64) -> dict:
    """Secondary workload: 64 prequantized Perlin fields, axes uniform in
    64..384, eb_rel in {1e-3, 1e-4, 1e-5} (seeds 1000+k), corrected by one
    msz_correct_batch launch (tile depths from the autotuner), against the same
    fields corrected by 64 separate msz_correct calls.  count < 64: the first
    count fields of that batch (profiling captures only)."""
    import torch

    from paper_2601_01787_gb300 import api, autotune, synth
    fields = synth.batch(64)[:count]
    n_tot = sum(fl.n for fl in fields)
    fs = [torch.from_numpy(fl.f).to(dev) for fl in fields]
    fhs = [torch.from_numpy(fl.fhat).to(dev) for fl in fields]
    xis = [fl.xi for fl in fields]
    caps = [fl.n // 4 for fl in fields]
    tz = autotune.tile_z_for([fl.shape for fl in fields], tune_missing=True)
    outs = [torch.empty_like(f) for f in fs]
    res = api.correct_batch(fs, fhs, xis, edit_capacities=caps, outs=outs, tile_z=tz, stream=stream)
    assert res.status == api.OK and all(r.status == api.OK for r in res.fields)

    def timed(fn):
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b)
            best = t if best is None else min(best, t)
        return best

    for _ in range(2):
        api.correct_batch(fs, fhs, xis, edit_capacities=caps, outs=outs, tile_z=tz, stream=stream)
    t_batch = timed(lambda: api.correct_batch(fs, fhs, xis, edit_capacities=caps, outs=outs, tile_z=tz,
                                              stream=stream))
    # the same launch captured once in a CUDA graph and replayed
    plan = api.BatchPlan(fs, fhs, xis, edit_capacities=caps, outs=outs, tile_z=tz, stream=stream)
    graph = plan.graph()
    graph.replay()
    torch.cuda.synchronize()
    rg = plan.collect()
    assert rg.status == api.OK and all(r.status == api.OK for r in rg.fields)
    assert all(a.edit_count == b.edit_count for a, b in zip(rg.fields, res.fields))
    t_graph = timed(graph.replay)
    plan.close()
    ws1 = api.workspace(max(api.workspace_size(f.shape) for f in fs), dev)

    def singles():
        for k in range(len(fs)):
            api.correct(fs[k], fhs[k], xis[k], out=outs[k], edit_capacity=caps[k], ws=ws1, stream=stream)

    singles()
    t_single = timed(singles)
    # roofline of the batch kernel: the same operation and byte counts as the
    # single-field kernel, summed over the fields (their sweep logs and
    # uncertified counts from one more launch)
    rl = api.correct_batch(fs, fhs, xis, edit_capacities=caps, outs=outs, tile_z=tz, stream=stream,
                           log_capacity=64)
    ops = sum(algorithmic_alu_ops(fl.n, r.sweep_log, r.stats["uncertified"]) for fl, r in zip(fields, rl.fields))
    nbytes = sum(algorithmic_bytes(fl.n, r.sweep_log, r.edit_count, r.stats["uncertified"])
                 for fl, r in zip(fields, rl.fields))
    alu_pk = alu_peak(sm_mhz or 2070.0) / 1e9
    peak, peak_kind = load_peaks()
    t_s = t_batch * 1e-3
    roof = {"bound": "alu", "kernel": "k_batch_codes + k_batch", "ops": ops, "achieved": round(ops / t_s / 1e9, 1),
            "peak": round(alu_pk, 1), "unit": "Gop/s", "frac": round(ops / t_s / 1e9 / alu_pk, 4),
            "hbm": {"algorithmic_bytes": nbytes, "achieved": round(nbytes / t_s / 1e9, 1), "peak": peak,
                    "unit": "GB/s", "frac": round(nbytes / t_s / 1e9 / peak, 4), "peak_kind": peak_kind,
                    "traffic": traffic_record("k_batch_perlin64_traffic.json", "msz_batch.cu") if count == 64
                    else None}}
    what = "batch of 64" if count == 64 else f"first {count} fields of the batch of 64"
    return {"workload": f"perlin3d_prequant {what}, axes U{{64..384}}, eb_rel in {{1e-3,1e-4,1e-5}}, seeds 1000+k",
            "n_vertices": n_tot, "unit": UNIT, "value": round(n_tot / (t_batch * 1e-3) / 1e9, 4),
            "ms": round(t_batch, 4), "graph_replay_ms": round(t_graph, 4),
            "graph_replay_value": round(n_tot / (t_graph * 1e-3) / 1e9, 4), "separate_calls_ms": round(t_single, 4),
            "separate_calls_value": round(n_tot / (t_single * 1e-3) / 1e9, 4),
            "max_sweeps_over_fields": max(r.stats["sweeps"] for r in res.fields),
            "tile_z": sorted(set(tz)), "launches": 2, "roofline": roof}


def run_learned(dev, stream, reps: int = 3) -> dict:
    """The learned proposal against the plain loop on a 512^3 Gaussian-peak
    field (5000 peaks: the peak density of the 1024 x 1024 x 512 workload;
    seed 7; relative bound 1e-4; uniform noise): wall time on the device from
    f and fhat resident to a corrected field and its edit list, sweeps, and
    the verification of both results.  The network is trained first by its
    recipe (200 seeded 128^3 triples) unless the library's cache
    already holds it."""
    import torch

    from paper_2601_01787_gb300 import api, learned, synth
    net, info = learned.default_net(dev)
    fl = synth.peaks3d((512, 512, 512), seed=7, eb_rel=1e-4, npeaks=5000)
    f = torch.from_numpy(fl.f).to(dev)
    fh = torch.from_numpy(fl.fhat).to(dev)
    cap = fl.n // 2
    out = torch.empty_like(f)
    eidx = torch.empty(cap, dtype=torch.int32, device=dev)
    edel = torch.empty(cap, dtype=torch.float32, device=dev)
    kw = dict(out=out, edit_idx=eidx, edit_delta=edel, edit_capacity=cap, stream=stream)

    def timed(fn):
        best, res = None, None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            res = fn()
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b)
            best = t if best is None else min(best, t)
        return best, res

    timed(lambda: api.correct(f, fh, fl.xi, **kw))
    t_plain, rp = timed(lambda: api.correct(f, fh, fl.xi, **kw))
    assert rp.status == api.OK, api.status_str(rp.status)
    vp = api.verify(f, out)
    stream_plain = edit_stream(fh, out, eidx, rp.edit_count, stream)
    dense = dense_sweeps(api.correct(f, fh, fl.xi, log_capacity=1024, **kw), fl.n)
    timed(lambda: learned.correct_learned(f, fh, fl.xi, net, **kw))
    t_learned, rl = timed(lambda: learned.correct_learned(f, fh, fl.xi, net, **kw))
    assert rl.result.status == api.OK, api.status_str(rl.result.status)
    vl = api.verify(f, out)
    n = fl.n
    convs = time_convs(net, f, fh, fl.xi, stream)
    peak = load_bf16_peak()
    c32 = convs["conv32x32_relu"]
    return {"workload": "peaks3d_512x512x512: 5000 Gaussian peaks on Poisson(5) counts, seed 7, eb_rel 1e-4, "
                        "fhat = f + U[-xi, xi]",
            "n_vertices": n, "unit": UNIT, "shift": learned.SHIFT,
            "plain": {"ms": round(t_plain, 4), "value": round(n / (t_plain * 1e-3) / 1e9, 4),
                      "sweeps": rp.stats["sweeps"], "first_distorted": rp.stats["first_distorted"],
                      "edited": rp.edit_count, "kernel_ms": round(rp.stats["kernel_ns"] / 1e6, 4),
                      "verified": bool(vp["codes_equal"] and vp["wrong_labels"] == 0),
                      "edit_stream": stream_plain, "dense_sweeps": dense},
            "learned": {"ms": round(t_learned, 4), "value": round(n / (t_learned * 1e-3) / 1e9, 4),
                        "propose_ms": round(rl.propose_ms, 4),
                        "loop_kernel_ms": round(rl.from_g0.stats["kernel_ns"] / 1e6, 4),
                        "sweeps": rl.from_g0.stats["sweeps"], "first_distorted": rl.from_g0.stats["first_distorted"],
                        "edited": rl.result.edit_count, "fallback_to_plain": rl.fallback,
                        "verified": bool(vl["codes_equal"] and vl["wrong_labels"] == 0)},
            "convs": convs,
            "conv_roofline": {"bound": "tensor", "kernel": "k_conv<32,32,RELU>", "achieved": c32["tflops"],
                              "peak": peak[0], "unit": "TFLOP/s", "frac": round(c32["tflops"] / peak[0], 4),
                              "peak_kind": peak[1], "flops_per_voxel": conv_flops_per_voxel(32, 32)},
            "training": {"recipe": learned.RECIPE | {"shape": list(learned.RECIPE["shape"])},
                         "cached": info["cached"], "train_s": None if info.get("train_s") is None else
                         round(info["train_s"], 2), "final_loss": info.get("final_loss")}}


def dense_sweeps(res, n: int) -> dict | None:
    """The whole-grid detection sweeps of a correction (from its sweep log
    and device timeline): their mean device time and HBM rate.  Compulsory
    bytes of one: read g (4 B/vertex, staged by TMA), read the uncertified
    bitmap and clear the worklist bitmap (N/8 B each), read the codes of f of
    the uncertified vertices (1 B each)."""
    log, tl = res.sweep_log, res.timeline
    ms = []
    for k in range(1, len(log)):
        if int(log[k, 0]) == n and tl[k][0] > 0 and tl[k - 1][1] > 0:
            ms.append((tl[k][0] - tl[k - 1][1]) / 1e6)
    if not ms:
        return None
    peak, kind = load_peaks()
    nbytes = 4 * n + 2 * (n // 8) + int(res.stats["uncertified"])
    mean = sum(ms) / len(ms)
    gbs = nbytes / (mean * 1e-3) / 1e9
    return {"count": len(ms), "ms_mean": round(mean, 4), "algorithmic_bytes": nbytes, "gbs": round(gbs, 1),
            "frac_of_hbm": round(gbs / peak, 4), "peak_kind": kind}


def edit_stream(fh, g, eidx, count: int, stream, reps: int = 3) -> dict:
    """The edit list of a corrected field as an encoded stream
    (msz_edits_encode): its length against the raw 8-byte (index, delta)
    pairs, and the device time of encoding it and of decoding it onto a copy
    of fhat (checked to give back g bit for bit)."""
    import torch

    from paper_2601_01787_gb300 import api
    fh1, g1, idx = fh.reshape(-1), g.reshape(-1), eidx[:count]
    field = torch.empty_like(fh1)

    def timed(fn):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            res = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, res

    enc_ms, s = timed(lambda: api.encode_edits(fh1, g1, idx, stream=stream))

    def dec():
        field.copy_(fh1)
        return api.decode_edits(s, field, stream=stream)

    dec_ms, got = timed(dec)
    exact = got == count and torch.equal(field.view(torch.int32), g1.view(torch.int32))
    nbytes = int(s.numel())
    # compulsory bytes: encoding reads the indices (4 B), fhat and g at them
    # (8 B) and writes the stream; decoding reads the stream and rewrites the
    # field at the indices (8 B) -- plus the copy of fhat the timing includes
    enc_b = 12 * count + nbytes
    dec_b = nbytes + 8 * count + 8 * fh1.numel()
    peak, kind = load_peaks()
    enc_gbs, dec_gbs = enc_b / (enc_ms * 1e-3) / 1e9, dec_b / (dec_ms * 1e-3) / 1e9
    return {"edits": count, "bytes": nbytes, "bytes_per_edit": round(nbytes / max(count, 1), 4),
            "raw_bytes_per_edit": 8, "ratio_vs_raw": round(8 * count / max(nbytes, 1), 3),
            "encode_ms": round(enc_ms, 4), "decode_ms": round(dec_ms, 4), "decode_exact": bool(exact),
            "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_kind": kind,
                         "encode": {"algorithmic_bytes": enc_b, "achieved": round(enc_gbs, 1),
                                    "frac": round(enc_gbs / peak, 4)},
                         "decode_with_fhat_copy": {"algorithmic_bytes": dec_b, "achieved": round(dec_gbs, 1),
                                                   "frac": round(dec_gbs / peak, 4)}}}


def conv_flops_per_voxel(cin: int, cout: int) -> int:
    """Dense FLOPs of one 3x3x3 conv layer per output voxel (padded channels)."""
    return 2 * 27 * cin * cout


def time_convs(net, f, fh, xi, stream, reps: int = 5) -> dict:
    """Device time of each conv layer of the proposal on this field (CUDA
    events on the launching stream, after one warm-up launch each)."""
    import torch

    from paper_2601_01787_gb300 import learned
    n = f.numel()
    x0 = learned.features(f, fh, xi, stream=stream)
    net.build_images(stream=stream)
    a = torch.empty(n, 32, dtype=torch.bfloat16, device=f.device)
    b = torch.empty_like(a)
    g0 = torch.empty_like(f)
    layers = [("conv16x32_relu", lambda: learned.conv(x0, 16, 32, learned.MODE_RELU, f.shape, net._img[0], net.err,
                                                      bias=net.b[0], out_bf16=a, stream=stream), 16, 32),
              ("conv32x32_relu", lambda: learned.conv(a, 32, 32, learned.MODE_RELU, f.shape, net._img[1], net.err,
                                                      bias=net.b[1], out_bf16=b, stream=stream), 32, 32),
              ("conv32x16_head", lambda: learned.conv(b, 32, 16, learned.MODE_HEAD, f.shape, net._img[3], net.err,
                                                      bias=net.b[3], f=f, fhat=fh, xi=xi, g0=g0, stream=stream),
               32, 16)]
    out = {}
    for name, fn, cin, cout in layers:
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": round(ms, 4), "tflops": round(n * conv_flops_per_voxel(cin, cout) / (ms * 1e-3) / 1e12, 2)}
    net.check()
    return out


def profile_conv(args) -> None:
    """Profiling case (captures only): two proposals on a small Gaussian-peak
    field with an untrained network (the weights do not change the work)."""
    import torch

    from paper_2601_01787_gb300 import learned, synth
    fl = synth.peaks3d(SHAPE, seed=7, eb_rel=1e-4)
    f = torch.from_numpy(fl.f).cuda()
    fh = torch.from_numpy(fl.fhat).cuda()
    net = learned.ProposalNet(seed=1)
    for _ in range(2):
        net.propose(f, fh, fl.xi)
    torch.cuda.synchronize()
    net.check()
    print(json.dumps({"profile_conv": list(SHAPE)}))


def api_source_hash() -> str:
    """Identity of the correction kernel's sources and flags (the traffic
    record applies only while it is unchanged)."""
    from paper_2601_01787_gb300 import _build
    return _build.unit_hash("msz_correct.cu")


def traffic_record(name: str, unit: str):
    """DRAM bytes (read + write) of one launch from the ncu record
    profiles/<name>, or None unless the record was taken of the kernels
    translation unit `unit` builds now (same code hash)."""
    from paper_2601_01787_gb300 import _build
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    return rec.get("traffic_bytes") if rec.get("unit_hash") == _build.unit_hash(unit) else None


def link_reference(hf, hfh, f, fh, stream, reps: int = 5) -> dict:
    """The host link measured in the same run: one step's inputs (f and fhat,
    pinned) copied to the device by plain cudaMemcpyAsync calls, timed with
    CUDA events -- on one stream, and split in halves over two streams."""
    import torch
    nbytes = hf.numel() * 4 + hfh.numel() * 4

    def one_stream():
        f.copy_(hf, non_blocking=True)
        fh.copy_(hfh, non_blocking=True)

    side = torch.cuda.Stream(device=f.device)

    def two_streams():
        side.wait_stream(stream)
        f.copy_(hf, non_blocking=True)
        with torch.cuda.stream(side):
            fh.copy_(hfh, non_blocking=True)
        stream.wait_stream(side)

    out = {"bytes": nbytes, "api": "cudaMemcpyAsync from pinned host memory (torch copy_, non_blocking)"}
    for name, fn in (("h2d_gbs", one_stream), ("h2d_two_streams_gbs", two_streams)):
        with torch.cuda.stream(stream):
            fn()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
        torch.cuda.synchronize()
        out[name] = round(nbytes * reps / (a.elapsed_time(b) * 1e-3) / 1e9, 2)
    return out


# ------------------------------------------------------------ CPU oracle
def cpu_baseline(fl, slab: int) -> dict:
    """The CPU oracle, as it stands (single thread), on the first `slab` z-planes
    of the same field and bound."""
    import oracle
    f = np.ascontiguousarray(fl.f[:slab])
    fh = np.ascontiguousarray(fl.fhat[:slab])
    oracle.build()
    t0 = time.perf_counter()
    r = oracle.correct(f, fh, fl.xi)
    dt = time.perf_counter() - t0
    assert r.status == oracle.OK
    return {"value": round(f.size / dt / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {slab} z-planes of the {workload_name()} workload ({f.size} vertices), worklist mode",
            "seconds": round(dt, 3), "sweeps": r.sweeps}


def cpu_baseline_configs() -> dict:
    """The CPU oracle (single thread) on the two configurations of
    run_configs: the whole 2D field, and the first 8 z-planes of the peak
    field (a bounded sample: the whole field takes about 14 minutes)."""
    import oracle

    from paper_2601_01787_gb300 import synth
    out = {}
    fl = synth.perlin2d((256, 256), seed=1, eb_rel=1e-3)
    for name, f, fh in (("perlin2d_256x256, the whole field", fl.f, fl.fhat),):
        t0 = time.perf_counter()
        r = oracle.correct(np.ascontiguousarray(f), np.ascontiguousarray(fh), fl.xi)
        dt = time.perf_counter() - t0
        out[name] = {"value": round(f.size / dt / 1e9, 6), "unit": UNIT, "seconds": round(dt, 3), "sweeps": r.sweeps}
    fl = synth.peaks3d((512, 1024, 1024), seed=3, eb_rel=1e-4)
    f, fh = np.ascontiguousarray(fl.f[:8]), np.ascontiguousarray(fl.fhat[:8])
    t0 = time.perf_counter()
    r = oracle.correct(f, fh, fl.xi)
    dt = time.perf_counter() - t0
    out["peaks3d_1024x1024x512, first 8 z-planes"] = {"value": round(f.size / dt / 1e9, 6), "unit": UNIT,
                                                      "seconds": round(dt, 3), "sweeps": r.sweeps}
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    from paper_2601_01787_gb300 import synth
    fl = synth.perlin3d_prequant(SHAPE, seed=SEED, eb_rel=EB_REL)
    slab = args.ref_slab
    f = np.ascontiguousarray(fl.f[:slab])
    fh = np.ascontiguousarray(fl.fhat[:slab])
    oracle.build()
    for _ in range(args.warmup):
        oracle.correct(f, fh, fl.xi)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.correct(f, fh, fl.xi)
        times.append(time.perf_counter() - t0)
        assert r.status == oracle.OK
    ms = statistics.mean(times) * 1e3
    value = f.size / (ms * 1e-3) / 1e9
    sample = f"first {slab} z-planes of the {workload_name()} workload ({f.size} vertices), worklist mode"
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(fl.n),
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-field batch measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal comparison")
    ap.add_argument("--no-large", dest="large", action="store_false",
                    help="skip the 1024^3 field (about 10 s of the run)")
    ap.add_argument("--no-relaxed", action="store_true", help="skip the relaxed-synchronization comparison")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the 2D 256^2 field and the 1024x1024x512 peak field (about 20 s of the run)")
    ap.add_argument("--cpu-slab", type=int, default=128, help="z-planes of the CPU-baseline sample")
    ap.add_argument("--ref-slab", type=int, default=24, help="z-planes per reference-arm step")
    ap.add_argument("--shape", default=None, help="nz,ny,nx of a smaller field (profiling captures only)")
    ap.add_argument("--batch-fields", type=int, default=64,
                    help="the first N fields of the 64-field batch (profiling captures only)")
    ap.add_argument("--profile-conv", action="store_true",
                    help="run two learned proposals on a --shape peak field and exit (profiling captures only)")
    args = ap.parse_args(argv)
    if args.shape:
        global SHAPE
        SHAPE = tuple(int(v) for v in args.shape.split(","))
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if not 1 <= args.batch_fields <= 64:
        ap.error("--batch-fields must be in 1..64")
    if args.profile_conv:
        profile_conv(args)
        return
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, ws, rank)
        else:
            run_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
