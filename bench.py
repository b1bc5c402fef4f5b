#!/usr/bin/env python
"""Benchmark of the GB300 radar chain (SAT + 2D CA-CFAR, paper Sec. II).

One JSON line on stdout (rank 0). A step is one pass of the whole hot path --
fast-time detrend, slow-time mean filter and normalisation, band DFT
magnitude, summed-area table and SAT CA-CFAR -- over one 1024 x 4096 raw frame
(8 targets, training 16 / guard 4 cells per side, Pfa 1e-6). Frames come from
a ring of 16 distinct seeded frames resident in HBM (268 MB, larger than the
129 MB L2), so every step reads its frame from HBM.

Also reported: SAT+CFAR Gcells/s on an 8192 x 8192 square-law map (the HBM
roofline case), per-kernel device times from the library's CUDA-event trace,
the end-to-end rate through the public API with host buffers, the CPU oracle's
rate on the host cores, and SM clocks sampled during the timed region.

  python bench.py [--steps K] [--warmup W] [--impl ours|reference]
  torchrun --nproc-per-node N bench.py --gpus N ...   (N independent replicas)
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DTYPE = ("f32 (band DFT: y as integer + FP16 head + tail, twiddles x 2^9 as integer + FP16 head + tail, six FP16 "
         "products with the integer x integer one accumulated exactly, FP32 accumulation; SAT + CFAR: exact 64-bit "
         "fixed point)")
METRIC = "SAT+CA-CFAR Gcells/s and full-chain frames/s at 1 GB300; % HBM roofline; p99 latency"
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu --set full capture
# of each kernel as it stands (summaries in profiles/): k_band_dft_tma on the 1024x4096 frame
# (bench.py --profile chain); the I64 table kernels and k_cfar_ring on a 4096x4096 map (bench.py
# --profile map), times 4 for the 8192x8192 map; k_sat_cfar_stream_tma on a 6144x6144 map (bench.py
# --profile fused --map-size 6144), times (8192/6144)^2 (their traffic grows with the cells).
TRAFFIC = {"band_dft": 32.43e6, "sat_i64_8192": 4 * 222.3e6, "cfar_ring_8192": 4 * 220.2e6,
           "sat_cfar_stream_8192": 319.1e6}
RING = 16
MIN_TIMED_MS = 250.0  # device time the headline is timed over, whatever K is


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-map", action="store_true", help="skip the 8192^2 SAT+CFAR measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-frame mixed batch measurement")
    ap.add_argument("--profile", choices=["chain", "map", "batch", "fused", "os"],
                    help="run one small fixed case a few times for a profiler capture and exit (no JSON line): "
                         "chain = the 1024x4096 frame through the per-frame calls, map = SAT (I64) + CFAR on a "
                         "--map-size square map, batch = one 64-frame mixed batch")
    ap.add_argument("--map-size", type=int, default=4096)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-frames", type=int, default=2000,
                    help="frames of the paced serving run (200 frames/s offered); 10000 = the full stream")
    ap.add_argument("--serve-burst", type=int, default=10000, help="frames of the time-compressed serving run")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers
def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"], "sm_max_mhz": d.get("sm_max_mhz", 2070.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled during the timed region.

    Reads NVML through ctypes every 0.5 ms on a background thread (read-only
    queries; no setting is changed); falls back to nvidia-smi at 200 ms.
    """

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device_index: int):
        self.dev = device_index
        self.samples, self.reasons = [], set()
        self.max_mhz = None
        self.thread = None
        self.proc = None
        self.lib = None
        try:
            import ctypes
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(device_index), ctypes.byref(h)) != 0:
                raise OSError("no NVML handle")
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) == 0:
                self.max_mhz = float(mx.value)
            self.lib, self.h, self.ct = lib, h, ctypes
        except Exception:
            self.lib = None

    def _loop(self):
        import time as _t
        ct, lib, h = self.ct, self.lib, self.h
        clk, rs = ct.c_uint(), ct.c_ulonglong()
        reason_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        while self.running:
            if lib.nvmlDeviceGetClockInfo(h, ct.c_int(1), ct.byref(clk)) == 0:
                self.samples.append(float(clk.value))
            if reason_fn(h, ct.byref(rs)) == 0:
                for bit, name in self.REASONS.items():
                    if rs.value & bit:
                        self.reasons.add(name)
            _t.sleep(0.0005)

    def start(self):
        if self.lib is not None:
            import threading
            self.running = True
            self.thread = threading.Thread(target=self._loop, daemon=True)
            self.thread.start()
            return
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=clocks.sm,clocks.max.sm,"
                                          "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                                          "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.running = False
            self.thread.join()
            return {"sm_mhz": statistics.median(self.samples) if self.samples else None,
                    "sm_max_mhz": self.max_mhz, "reasons": sorted(self.reasons), "samples": len(self.samples),
                    "source": "nvml"}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock source"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax = [], []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 6:
                    continue
                try:
                    sm.append(float(p[0]))
                    smax.append(float(p[1]))
                except ValueError:
                    continue
                for n, v in zip(names, p[2:6]):
                    if v.lower() == "active":
                        self.reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(self.reasons), "samples": len(sm), "source": "nvidia-smi"}


def dist_setup():
    from paper_2012_11077_gb300 import replicas
    return replicas.setup()


def max_over_ranks(x: float, dist) -> float:
    from paper_2012_11077_gb300 import replicas
    return replicas.max_over_ranks(x, dist)


def barrier(dist):
    from paper_2012_11077_gb300 import replicas
    replicas.barrier(dist)


# ---------------------------------------------------------------- CPU oracle timing
def oracle_rate(budget_s: float = 10.0, max_frames: int = 50):
    """Frames/s of the FP64 oracle chain on this host (bounded sample)."""
    import oracle
    import synth
    case = synth.large_frame_case(0)
    w = case.window
    X = synth.radar_frame(case.spec)
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.run_chain(X, synth.FS_HZ, case.mean_len, w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= max_frames:
            break
    return n / el, n, el


def oracle_rate_single_core(budget_s: float = 8.0, max_frames: int = 10):
    """The same on one core: a child process with every BLAS / OpenMP pool at one thread."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_rate(%r, %d)))" % (ROOT, budget_s, max_frames))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
        v, n, el = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": v, "unit": "frames/s", "cores": 1,
                "sample": f"{n} frames of 1024x4096 in {el:.1f} s, numpy FP64, one thread"}
    except Exception as e:  # the single-core figure is context only
        return {"value": None, "unit": "frames/s", "cores": 1, "error": str(e)[:200]}


def reference_arm(args, rank):
    if rank != 0:
        return
    import synth
    import oracle
    case = synth.large_frame_case(0)
    w = case.window
    X = synth.radar_frame(case.spec)

    def step():
        oracle.run_chain(X, synth.FS_HZ, case.mean_len, w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)

    t_w = time.perf_counter()
    for _ in range(max(1, args.warmup)):
        step()
    t_step = (time.perf_counter() - t_w) / max(1, args.warmup)
    # a bounded sample: at most about two minutes of oracle work (at least 3 frames)
    n = max(3, min(args.steps, int(120.0 / max(t_step, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(n):
        step()
    el = time.perf_counter() - t0
    v = n / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded UWB radar frame)",
            "config": {"workload": "full chain, one 1024x4096 raw frame per step (8 targets, training 16, "
                                   "guard 4, Pfa 1e-6, mean filter 5, fs 20 Hz)"},
            "cpu_baseline": {"value": v, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{n} of the {args.steps} steps' frames of 1024x4096 timed (at most about "
                                       f"120 s of oracle work), numpy FP64 (BLAS threads = all cores)"},
            "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- batching
def sat_mode_name(rc, mode: int) -> str:
    return {rc.RCFAR_SAT_I64: "I64 (streaming CFAR)", rc.RCFAR_SAT_TILE_I64: "TILE_I64",
            rc.RCFAR_SAT_FUSED: "FUSED (streaming SAT + CFAR)"}.get(mode, str(mode))


def batch_measure(rc, torch, synth, local, rank, n_frames=64, reps=10):
    """64 frames of uneven size and window: one rcfar_run_batch (graph-captured)
    against looping the per-frame path (rcfar_preprocess, rcfar_sat,
    rcfar_cfar) over the same frames; both produce the same decisions."""
    cases = synth.mixed_batch_cases(n_frames, seed=100 + rank)
    params = rc.make_pre_params(synth.FS_HZ, mean_len=5, halo_c=-1)
    h = rc.rcfar_create(device=local, max_rows=1024, max_cols=1024, max_n=4096, max_window=32,
                        max_frames=n_frames, batch_bytes=3 << 30)
    frames, descs, dets, single = [], [], [], []
    samples = 0
    for c in cases:
        x = torch.from_numpy(synth.radar_frame(c.spec)).cuda()
        w = c.window
        win = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
        p1 = rc.make_pre_params(synth.FS_HZ, mean_len=5, halo_c=w.train_c + w.guard_c)
        band = rc.rcfar_band_plan(c.spec.N, p1)
        det = torch.empty((c.spec.M, band.cols), dtype=torch.uint8, device="cuda")
        det1 = torch.empty_like(det)
        P1 = torch.empty((c.spec.M, band.cols), dtype=torch.float32, device="cuda")
        frames.append(x)
        dets.append(det)
        descs.append(rc.frame_desc(x, win, det))
        single.append((x, p1, band, win, det1, P1))
        samples += c.spec.M * c.spec.N
    rc.rcfar_prepare(h, descs, params)

    def per_frame():
        for x, p1, band, win, det1, P1 in single:
            rc.rcfar_preprocess(h, x, p1, P1)
            v = rc.rcfar_sat(h, P1, value_bound=band.value_bound, mode=rc.RCFAR_SAT_TILE_I64)
            rc.rcfar_cfar(h, v, P1, win, band.k_lo - band.c0, band.k_hi - band.c0, det1)

    def batched():
        rc.rcfar_run_batch(h, descs, params)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, n):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    t_single = timed(per_frame, reps)
    # the same per-frame calls captured once into a CUDA graph (no host launch
    # work per frame): the fairer denominator for the batch's speed-up
    t_single_graph = None
    try:
        sg = torch.cuda.Stream()
        gpf = torch.cuda.CUDAGraph()
        with torch.cuda.stream(sg):
            per_frame()
            sg.synchronize()
            with torch.cuda.graph(gpf, stream=sg):
                per_frame()
        torch.cuda.synchronize()
        t_single_graph = timed(gpf.replay, reps)
    except Exception as ex:  # capture refused: report the eager baseline only
        print(f"per-frame graph capture failed: {ex}", file=sys.stderr)
    # the library's autotuner picks the batch schedule (results are the same for every schedule)
    tuning = rc.rcfar_tune_batch(h, descs, params, reps=3)
    t_batch_eager = timed(batched, reps)
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        batched()
        stream.synchronize()
        with torch.cuda.graph(g, stream=stream):
            batched()
    torch.cuda.synchronize()
    t_batch = timed(g.replay, reps)
    rc.rcfar_trace_enable(h, True)
    batched()
    tr = rc.rcfar_trace_read(h)
    rc.rcfar_trace_enable(h, False)
    per_frame()
    g.replay()
    torch.cuda.synchronize()
    same = all(torch.equal(d, s[4]) for d, s in zip(dets, single))
    ok = rc.rcfar_get_error(h) == rc.RCFAR_OK
    rc.rcfar_destroy(h)
    return {"frames": n_frames, "workload": "64 frames, M ~ U{128..1024}, N ~ U{256..4096}, training {4,8,16}, "
                                            "guard {1,2,4}, Pfa {1e-3,1e-4,1e-6}, 0-10 targets",
            "batched_frames_per_s": n_frames / (t_batch * 1e-3),
            "batched_eager_frames_per_s": n_frames / (t_batch_eager * 1e-3),
            "per_frame_path_frames_per_s": n_frames / (t_single * 1e-3),
            "speedup_vs_per_frame": t_single / t_batch,
            "per_frame_graph_frames_per_s": n_frames / (t_single_graph * 1e-3) if t_single_graph else None,
            "speedup_vs_per_frame_graph": t_single_graph / t_batch if t_single_graph else None,
            "kernels_us": {k: 1e3 * t / n for k, (n, t) in tr.items()},
            "tuning": {"dft_kblocks_per_cta": tuning.dft_kblocks_per_cta,
                       "sat_mode": sat_mode_name(rc, tuning.sat_mode),
                       "cfar_tile": [tuning.cfar_tile_rows, tuning.cfar_tile_cols],
                       "candidates": tuning.candidates, "best_ms": tuning.best_ms},
            "samples_per_s": samples / (t_batch * 1e-3),
            "decisions_identical": bool(same and ok)}


def latency_small_frame(rc, torch, synth, local, n=400):
    """Latency of one 256 x 512 raw frame (2 targets, training 8 / guard 2,
    Pfa 1e-4) through the C ABI, from raw frame in HBM to decisions in HBM:
    rcfar_preprocess then rcfar_sat_cfar, issued eagerly or replayed as one
    CUDA graph. host_ms = wall time from the first call until the stream has
    finished (what a caller waits); device_ms = CUDA events around the work on
    the stream. Frames of this size are L2-resident: a latency case, not a
    bandwidth one."""
    case = synth.small_frame_case(0)
    w = case.window
    M, N = case.spec.M, case.spec.N
    params = rc.make_pre_params(synth.FS_HZ, mean_len=case.mean_len, halo_c=case.halo_c)
    band = rc.rcfar_band_plan(N, params)
    win = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
    h = rc.rcfar_create(device=local, max_rows=M, max_cols=256, max_n=N, max_window=32, max_frames=1)
    x = torch.from_numpy(synth.radar_frame(case.spec)).cuda()
    P = torch.empty((M, band.cols), dtype=torch.float32, device="cuda")
    det = torch.empty((M, band.cols), dtype=torch.uint8, device="cuda")

    def chain():
        rc.rcfar_preprocess(h, x, params, P)
        rc.rcfar_sat_cfar(h, P, band.value_bound, win, band.k_lo - band.c0, band.k_hi - band.c0, det, map_cut=False)

    for _ in range(10):
        chain()
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            chain()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": f"{M}x{N} raw frame, training {w.train_r} / guard {w.guard_r}, Pfa {w.pfa:g}, "
                       f"{band.cols}-bin band map", "samples": n}
    for name, fn in (("eager", chain), ("graph", g.replay)):
        for _ in range(10):
            fn()
        torch.cuda.synchronize()
        host, dev = [], []
        for _ in range(n):
            t0 = time.perf_counter()
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            host.append(1e3 * (time.perf_counter() - t0))
            dev.append(e0.elapsed_time(e1))
        host.sort()
        dev.sort()
        out[name] = {"host_ms_p50": host[n // 2], "host_ms_p99": host[int(0.99 * n)],
                     "device_ms_p50": dev[n // 2], "device_ms_p99": dev[int(0.99 * n)]}
    out["status"] = rc.status_string(rc.rcfar_get_error(h))
    rc.rcfar_destroy(h)
    return out


def precision_study(rc, torch, h, Pt, w):
    """Precision of the summed-area table's storage choices on one map (eq. 3),
    each against the exact path: the I64 table (64-bit fixed point, exact up
    to the map's quantisation; the GPU tests hold it to the FP64 oracle on
    this map). Modes: TILE_F32 (FP32 tile-local table with exact int64
    inter-tile carries), the map stored in FP16 (times a power of two so that
    its largest value fits) with an exact table, and a naive global FP32
    table. Per mode: the table entries' largest error relative to max(|S|, 1)
    (1 = the noise mean), the CUT
    thresholds' largest relative error, and the decisions that differ outside
    and inside the 1e-5 tie margin."""
    import math

    R, C = Pt.shape
    win = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
    bound = float(Pt.max().item())
    exp2 = int(math.ceil(math.log2(bound / 60000.0)))
    P16 = (Pt / 2.0 ** exp2).half()
    det = torch.empty((R, C), dtype=torch.uint8, device="cuda")
    thr = torch.empty((R, C), dtype=torch.float32, device="cuda")
    S = torch.empty((R, C), dtype=torch.float64, device="cuda")

    def run(mode, Pm, e2):
        # FP16 rounding can lift the largest value slightly above the float32 map's
        b = bound if e2 == 0 else max(bound, float(Pm.float().max()) * 2.0 ** e2)
        v = rc.rcfar_sat(h, Pm, value_bound=b, mode=mode, map_exp2=e2)
        rc.rcfar_cfar(h, v, Pm, win, 0, C - 1, det, thr, map_exp2=e2)
        rc.rcfar_sat_materialize(h, v, S)
        return rc.status_string(rc.rcfar_get_error(h))

    run(rc.RCFAR_SAT_I64, Pt, 0)
    S_ref, det_ref, thr_ref = S.clone(), det.clone(), thr.clone().double()
    cut = thr_ref > 0
    tie = cut & ((Pt.double() - thr_ref).abs() < 1e-5 * thr_ref)
    out = {"workload": f"{R}x{C} square-law map, 200 targets over 80 dB, training {w.train_r} / guard {w.guard_r}, "
                       f"Pfa {w.pfa:g}",
           "reference": "the exact I64 table path (held to the FP64 oracle by tests/test_gpu_precision.py)",
           "detections": int(det_ref.sum()), "near_ties": int(tie.sum())}
    for name, mode, Pm, e2 in (("TILE_F32", rc.RCFAR_SAT_TILE_F32, Pt, 0),
                               ("FP16_STORAGE", rc.RCFAR_SAT_TILE_I64, P16, exp2),
                               ("NAIVE_F32", rc.RCFAR_SAT_NAIVE_F32, Pt, 0)):
        st = run(mode, Pm, e2)
        diff = det != det_ref
        out[name] = {"status": st,
                     "sat_max_rel_err": float(((S - S_ref).abs() / S_ref.abs().clamp_min(1.0)).max()),
                     "thr_max_rel_err": float(((thr.double() - thr_ref).abs()[cut] / thr_ref[cut]).max()),
                     "mismatches_outside_margin": int((diff & ~tie).sum()),
                     "mismatches_inside_margin": int((diff & tie).sum())}
    out["FP16_STORAGE"]["map_exp2"] = exp2
    del S, S_ref, P16
    return out


# ---------------------------------------------------------------- our arm
def serving_measure(rc, torch, synth, local, rank, n_paced, n_burst):
    """Poisson stream from 32 drones (fixed frame size and window per drone,
    sizes and windows as in the mixed batch) through the library's serving loop
    (continuous batching, 8 GB device-memory admission budget, 3 batches in
    flight), in two request forms: frames in pinned host memory (copied in,
    decisions copied back: copies inside every latency) and frames already in
    device memory (read in place, decisions written to device buffers).
    Paced: frames submitted at their arrival times (200 frames/s offered):
    latency = completion - arrival, split into the wait for admission (arrival
    to admission) and the batch's service (admission to completion), with the
    host's own lateness in submitting (submission - arrival). Time-compressed:
    every frame submitted at once (one rcfar_server_submit_many burst):
    sustained frames/s."""
    params = rc.make_pre_params(synth.FS_HZ, mean_len=5, halo_c=-1)
    arrivals, drones, variants, cases = synth.serving_stream(n_requests=max(n_paced, n_burst), n_drones=32,
                                                             rate_hz=200.0, seed=7 + rank, n_variants=4)
    srv = rc.rcfar_server_create(device=local, budget_bytes=8 << 30, slots=3, max_batch_frames=64, max_rows=1024,
                                 max_n=4096, max_window=20, params=params)
    pool, pool_dev, cols = {}, {}, {}
    for d, vs in enumerate(cases):
        w = vs[0].window
        cols[d] = rc.rcfar_band_plan(vs[0].spec.N, rc.make_pre_params(synth.FS_HZ, mean_len=5,
                                                                      halo_c=w.train_c + w.guard_c)).cols
        for v, c in enumerate(vs):
            pool[(d, v)] = torch.from_numpy(synth.radar_frame(c.spec)).pin_memory()
            pool_dev[(d, v)] = pool[(d, v)].cuda()
    wins = [rc.make_window(vs[0].window.train_r, vs[0].window.train_c, vs[0].window.guard_r, vs[0].window.guard_c,
                           vs[0].window.pfa) for vs in cases]
    rc.rcfar_server_prepare(srv, [vs[0].spec.N for vs in cases], wins)
    # decision buffers: one arena per memory kind, a slice per request
    n_all = max(n_paced, n_burst)
    sizes = [pool[(int(drones[i]), int(variants[i]))].shape[0] * cols[int(drones[i])] for i in range(n_all)]
    arena = {"host": torch.empty(sum(sizes), dtype=torch.uint8).pin_memory(),
             "device": torch.empty(sum(sizes), dtype=torch.uint8, device="cuda")}
    torch.cuda.synchronize()
    offs = [0]
    for z in sizes:
        offs.append(offs[-1] + z)

    def det_of(i, mem):
        d = int(drones[i])
        return arena[mem][offs[i]:offs[i + 1]].view(pool[(d, 0)].shape[0], cols[d])

    def run(n, paced, mem):
        done, late = {}, []
        src = pool if mem == "host" else pool_dev
        gc.collect()
        gc.disable()  # a collection pause would count as the host's lateness in submitting
        if paced:
            t0 = rc.rcfar_server_now_ns() + 2_000_000
            for i in range(n):
                d, v = int(drones[i]), int(variants[i])
                t_arr = t0 + int(arrivals[i] * 1e9)
                while rc.rcfar_server_now_ns() < t_arr:
                    time.sleep(0.0001)
                late.append((rc.rcfar_server_now_ns() - t_arr) / 1e6)
                rc.rcfar_server_submit(srv, src[(d, v)], wins[d], det_of(i, mem), tag=i, arrival_ns=t_arr)
                if i % 32 == 31:
                    for c in rc.rcfar_server_poll(srv, 1024, 0):
                        done[c.tag] = c
        else:
            # the whole stream arrives at once: one burst through rcfar_server_submit_many
            reqs = [rc.server_request(src[(int(drones[i]), int(variants[i]))], wins[int(drones[i])],
                                      det_of(i, mem), tag=i) for i in range(n)]
            rc.rcfar_server_submit_many(srv, reqs)
        gc.enable()
        deadline = time.time() + 300
        while len(done) < n and time.time() < deadline:
            for c in rc.rcfar_server_poll(srv, 1024, 50):
                done[c.tag] = c
        bad = [c for c in done.values() if c.status != rc.RCFAR_OK]
        if len(done) < n or bad:
            raise RuntimeError(f"serving: {len(done)} of {n} completed, {len(bad)} failed")

        def pct(v):
            v = sorted(v)
            return {"p50_ms": v[len(v) // 2], "p99_ms": v[min(len(v) - 1, int(0.99 * len(v)))], "max_ms": v[-1]}

        cs = list(done.values())
        out = pct([(c.done_ns - c.arrival_ns) / 1e6 for c in cs])
        first = min(c.arrival_ns for c in cs)
        last = max(c.done_ns for c in cs)
        out.update({"frames": n, "frames_per_s": n / ((last - first) / 1e9),
                    "mean_batch": sum(c.batch_frames for c in cs) / n})
        if paced:
            out["admission_wait"] = pct([(c.admit_ns - c.arrival_ns) / 1e6 for c in cs])
            out["service"] = pct([(c.done_ns - c.admit_ns) / 1e6 for c in cs])
            out["host_submit_lateness"] = pct(late)
        return out

    res = {}
    for mem in ("host", "device"):
        run(min(256, n_all), False, mem)  # warm-up: every slot runs batches
        res[mem] = {"paced": run(n_paced, True, mem) if n_paced > 0 else None,
                    "time_compressed": run(n_burst, False, mem) if n_burst > 0 else None}
    st = rc.rcfar_server_get_stats(srv)
    rc.rcfar_server_destroy(srv)
    return {"workload": "Poisson stream, 32 drones (fixed size and window each, sizes M ~ U{128..1024}, "
                        "N ~ U{256..4096}), 200 frames/s offered; 8 GB budget, 3 slots",
            "host_memory": dict(res["host"], path="frames and decisions in pinned host memory (copies inside)"),
            "device_memory": dict(res["device"], path="frames already in HBM, decisions to HBM (no copies)"),
            "paced": res["host"]["paced"], "time_compressed": res["host"]["time_compressed"],
            "max_inflight_frames": st["max_inflight_frames"], "device_bytes": st["device_bytes"]}


def e2e_server(rc, torch, args, local, host_x, w, M, N, C, world, dist):
    """Full-chain frames/s from host buffers through rcfar_server_submit (the
    C-ABI call that takes host pointers): n frames submitted at once, timed
    from the first submission to the last completion (host clock)."""
    params = rc.make_pre_params(20.0, mean_len=5, halo_c=-1)
    win = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
    srv = rc.rcfar_server_create(device=local, budget_bytes=4 << 30, slots=3, max_batch_frames=8, max_rows=M,
                                 max_n=N, max_window=20, params=params)
    rc.rcfar_server_prepare(srv, [N], [win])
    n = max(4 * args.steps, 200)
    arena = torch.empty((n, M, C), dtype=torch.uint8).pin_memory()

    def run(count):
        t0 = rc.rcfar_server_now_ns()
        done = {}
        for i in range(count):
            rc.rcfar_server_submit(srv, host_x[i % len(host_x)], win, arena[i], tag=i)
            if i % 16 == 15:
                for c in rc.rcfar_server_poll(srv, 256, 0):
                    done[c.tag] = c
        deadline = time.time() + 120
        while len(done) < count and time.time() < deadline:
            for c in rc.rcfar_server_poll(srv, 256, 50):
                done[c.tag] = c
        if len(done) < count or any(c.status != rc.RCFAR_OK for c in done.values()):
            raise RuntimeError("e2e: frames missing or failed")
        return (max(c.done_ns for c in done.values()) - t0) / 1e9, done

    run(max(args.warmup, 3) * 8)
    barrier(dist)
    el, done = run(n)
    el = max_over_ranks(el, dist)
    st = rc.rcfar_server_get_stats(srv)
    rc.rcfar_server_destroy(srv)
    return {"value": world * n / el, "unit": "frames/s", "h2d_bytes_per_step": M * N * 4, "d2h_bytes_per_step": M * C,
            "h2d_gb_per_s": n * M * N * 4 / el / 1e9, "frames": n, "path": "rcfar_server_submit from pinned host memory, decisions back to pinned host memory; "
                                 "3 slots, batches of up to 8 frames",
            "mean_batch": sum(c.batch_frames for c in done.values()) / n, "device_bytes": st["device_bytes"]}


def ours(args, rank, world, local, dist):
    import numpy as np
    import torch

    import synth
    import paper_2012_11077_gb300 as rc
    from paper_2012_11077_gb300 import build as b

    torch.cuda.set_device(local)
    b.build()
    peaks = load_peaks()
    case = synth.large_frame_case(0)
    w = case.window
    M, N = case.spec.M, case.spec.N
    params = rc.make_pre_params(synth.FS_HZ, mean_len=case.mean_len, halo_c=case.halo_c)
    band = rc.rcfar_band_plan(N, params)
    C = band.cols
    win = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
    cut_lo, cut_hi = band.k_lo - band.c0, band.k_hi - band.c0
    h = rc.rcfar_create(device=local, max_rows=8192, max_cols=8192, max_n=N, max_window=32, max_frames=64,
                        batch_bytes=0)

    # ring of distinct frames in HBM (per rank: its own seeds)
    frames = []
    for i in range(RING):
        spec = synth.FrameSpec(M=M, N=N, n_targets=8, seed=1000 * rank + i)
        frames.append(torch.from_numpy(synth.radar_frame(spec)).cuda())
    maps = [torch.empty((M, C), dtype=torch.float32, device="cuda") for _ in range(RING)]
    dets = [torch.empty((M, C), dtype=torch.uint8, device="cuda") for _ in range(RING)]

    def chain(i):
        # SAT + CFAR fused (no table in device memory; decisions identical to rcfar_sat + rcfar_cfar)
        x, P, det = frames[i % RING], maps[i % RING], dets[i % RING]
        rc.rcfar_preprocess(h, x, params, P)
        rc.rcfar_sat_cfar(h, P, band.value_bound, win, cut_lo, cut_hi, det, map_cut=False)

    # warm-up (also builds the twiddle plan), then capture one graph per ring
    # slot and one graph of all RING consecutive steps (the same calls, frame
    # after frame: between two steps' kernels the programmatic launch then
    # overlaps set-up as it does within a step)
    for i in range(max(args.warmup, 3)):
        chain(i)
    torch.cuda.synchronize()
    assert rc.rcfar_get_error(h) == rc.RCFAR_OK
    stream = torch.cuda.Stream()
    graphs = []
    with torch.cuda.stream(stream):
        for i in range(RING):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                chain(i)
            graphs.append(g)
        ring_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(ring_graph, stream=stream):
            for i in range(RING):
                chain(i)
    torch.cuda.synchronize()
    for i in range(max(args.warmup, 3)):
        graphs[i % RING].replay()
    ring_graph.replay()
    torch.cuda.synchronize()

    # timed region: blocks of exactly K steps (K // RING replays of the ring's
    # graph, then K % RING one-step graphs), each bracketed by CUDA events on
    # the replay stream, repeated until at least MIN_TIMED_MS of device time
    # has been timed (a K of 20 steps alone is about a millisecond); the
    # median block is the step time
    clocks = ClockSampler(local)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    blocks_ms = []
    full, rem = divmod(args.steps, RING)
    while True:
        e0.record()
        for _ in range(full):
            ring_graph.replay()
        for j in range(rem):
            graphs[j].replay()
        e1.record()
        torch.cuda.synchronize()
        blocks_ms.append(e0.elapsed_time(e1))
        if sum(blocks_ms) >= MIN_TIMED_MS and len(blocks_ms) >= 3:
            break
    barrier(dist)
    ms = statistics.median(blocks_ms)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, dist)
    value = world * args.steps / (ms_max / 1e3)
    timing = {"blocks": len(blocks_ms), "steps_per_block": args.steps, "timed_ms_total": sum(blocks_ms),
              "block_ms_min": min(blocks_ms), "block_ms_median": ms, "block_ms_max": max(blocks_ms),
              "reported": "median block (exactly K steps) per rank, max over ranks",
              "submission": "CUDA graphs of %d consecutive frame steps (the remainder of a block one step per graph); "
                            "every step is one frame's rcfar_preprocess + rcfar_sat_cfar" % RING}
    assert rc.rcfar_get_error(h) == rc.RCFAR_OK

    def graph_rate(fn):
        """frames/s of fn(i) over the ring, captured as one CUDA graph of RING consecutive steps (as the
        headline) and replayed."""
        for i in range(3):
            fn(i)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            gv = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gv, stream=stream):
                for i in range(RING):
                    fn(i)
        torch.cuda.synchronize()
        gv.replay()
        torch.cuda.synchronize()
        reps = max(1, max(10, args.steps // 2) // RING)
        e0.record()
        for _ in range(reps):
            gv.replay()
        e1.record()
        torch.cuda.synchronize()
        assert rc.rcfar_get_error(h) == rc.RCFAR_OK
        return {"frames_per_s": reps * RING / (e0.elapsed_time(e1) / 1e3)}

    # the chain with the square-law detector and with per-range-bin z-score
    # normalisation (the next-step variants), captured and timed the same way
    variants = {}
    for vname, det_mode, norm_mode in (("square_law", 1, 0), ("row_zscore", 0, 1)):
        pv = rc.make_pre_params(synth.FS_HZ, mean_len=case.mean_len, halo_c=case.halo_c, detector=det_mode,
                                normalise=norm_mode)
        bv = rc.rcfar_band_plan(N, pv)

        def chain_v(i, pv=pv, bv=bv):
            x, P, det = frames[i % RING], maps[i % RING], dets[i % RING]
            rc.rcfar_preprocess(h, x, pv, P)
            rc.rcfar_sat_cfar(h, P, bv.value_bound, win, cut_lo, cut_hi, det, map_cut=False)

        variants[vname] = graph_rate(chain_v)

    # greatest-of / smallest-of thresholds on the same chain
    for vname, kind in (("greatest_of", rc.RCFAR_CFAR_GO), ("smallest_of", rc.RCFAR_CFAR_SO)):
        wk = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa, kind=kind)

        def chain_k(i, wk=wk):
            x, P, det = frames[i % RING], maps[i % RING], dets[i % RING]
            rc.rcfar_preprocess(h, x, params, P)
            rc.rcfar_sat_cfar(h, P, band.value_bound, wk, cut_lo, cut_hi, det, map_cut=False)

        variants[vname] = graph_rate(chain_k)

    # ordered-statistic thresholds on the same chain (an order statistic is not
    # a region sum: the map goes to the direct selection kernel)
    wos = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa, kind=rc.RCFAR_CFAR_OS)

    def chain_os(i):
        x, P, det = frames[i % RING], maps[i % RING], dets[i % RING]
        rc.rcfar_preprocess(h, x, params, P)
        rc.rcfar_cfar_direct(h, P, wos, cut_lo, cut_hi, det)

    variants["ordered_statistic"] = graph_rate(chain_os)

    # the paper's own frame size, 600 traces of 1024 range samples, given trace
    # by trace ([N][M], the acquisition order)
    pp = rc.make_pre_params(synth.FS_HZ, mean_len=case.mean_len, halo_c=case.halo_c,
                            x_layout=rc.RCFAR_X_TRACE_MAJOR)
    Np = 600
    bp = rc.rcfar_band_plan(Np, pp)
    xs_p = [torch.from_numpy(np.ascontiguousarray(
        synth.radar_frame(synth.FrameSpec(M=M, N=Np, n_targets=8, seed=5000 + 1000 * rank + i)).T)).cuda()
        for i in range(RING)]
    maps_p = [torch.empty((M, bp.cols), dtype=torch.float32, device="cuda") for _ in range(RING)]
    dets_p = [torch.empty((M, bp.cols), dtype=torch.uint8, device="cuda") for _ in range(RING)]

    def chain_p(i):
        rc.rcfar_preprocess(h, xs_p[i % RING], pp, maps_p[i % RING])
        rc.rcfar_sat_cfar(h, maps_p[i % RING], bp.value_bound, win, bp.k_lo - bp.c0, bp.k_hi - bp.c0,
                          dets_p[i % RING], map_cut=False)

    variants["paper_frame_1024x600_trace_major"] = graph_rate(chain_p)

    # the same 1024 x 4096 frames eight at a time through rcfar_run_batch (one
    # graph per batch, autotuned schedule): the throughput form of this workload
    hb = rc.rcfar_create(device=local, max_rows=M, max_cols=1024, max_n=N, max_window=32, max_frames=8,
                         batch_bytes=1 << 30)
    pbatch = rc.make_pre_params(synth.FS_HZ, mean_len=case.mean_len, halo_c=-1)
    dets_b = [torch.empty((M, C), dtype=torch.uint8, device="cuda") for _ in range(RING)]
    groups = [[rc.frame_desc(frames[j], win, dets_b[j]) for j in range(g0, g0 + 8)] for g0 in range(0, RING, 8)]
    rc.rcfar_prepare(hb, groups[0], pbatch)
    tuning_b = rc.rcfar_tune_batch(hb, groups[0], pbatch, reps=3)
    gb = []
    with torch.cuda.stream(stream):
        for grp in groups:
            rc.rcfar_run_batch(hb, grp, pbatch)
            stream.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                rc.rcfar_run_batch(hb, grp, pbatch)
            gb.append(g)
    torch.cuda.synchronize()
    for i in range(3):
        gb[i % len(gb)].replay()
    torch.cuda.synchronize()
    nb_rep = max(6, args.steps // 8)
    e0.record()
    for i in range(nb_rep):
        gb[i % len(gb)].replay()
    e1.record()
    torch.cuda.synchronize()
    assert rc.rcfar_get_error(hb) == rc.RCFAR_OK
    for i in range(RING):
        chain(i)
    torch.cuda.synchronize()
    chain_batched = {"frames_per_batch": 8, "frames_per_s": 8 * nb_rep / (e0.elapsed_time(e1) / 1e3),
                     "decisions_identical_to_per_frame": all(torch.equal(dets_b[j], dets[j]) for j in range(RING)),
                     "tuning": {"dft_kblocks_per_cta": tuning_b.dft_kblocks_per_cta,
                                "sat_mode": sat_mode_name(rc, tuning_b.sat_mode),
                                "best_ms": tuning_b.best_ms}}
    rc.rcfar_destroy(hb)

    # per-kernel device times (eager launches bracketed by CUDA events)
    rc.rcfar_trace_enable(h, True)
    for i in range(args.steps):
        chain(i)
    trace = rc.rcfar_trace_read(h)
    rc.rcfar_trace_enable(h, False)
    step_kernels = {k: {"launches": n, "avg_us": 1e3 * t / n} for k, (n, t) in trace.items()}
    # our kernels per chain step (the trace brackets every launch of the library)
    launches_per_step = round(sum(n for n, _ in trace.values()) / args.steps)
    # SAT + CFAR on the chain's band map: split (table in HBM) against fused
    P0, d0 = maps[0], dets[0]
    d1 = torch.empty_like(d0)

    def split_sc():
        v = rc.rcfar_sat(h, P0, value_bound=band.value_bound, mode=rc.RCFAR_SAT_TILE_I64)
        rc.rcfar_cfar(h, v, None, win, cut_lo, cut_hi, d1)

    def fused_sc():
        rc.rcfar_sat_cfar(h, P0, band.value_bound, win, cut_lo, cut_hi, d0, map_cut=False)

    def direct_sc():  # the cell-by-cell CA-CFAR the SAT replaces (Table I's "CA-CFAR")
        rc.rcfar_cfar_direct(h, P0, win, cut_lo, cut_hi, d1)

    def os_sc():
        rc.rcfar_cfar_direct(h, P0, wos, cut_lo, cut_hi, d1)

    chain_map = {}
    for nm, fn in (("direct_us", direct_sc), ("os_us", os_sc), ("split_us", split_sc), ("fused_us", fused_sc)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(20):
            fn()
        e1.record()
        torch.cuda.synchronize()
        chain_map[nm] = 1e3 * e0.elapsed_time(e1) / 20
    chain_map["decisions_identical"] = bool(torch.equal(d0, d1))
    chain_map["map"] = f"{M}x{C} band map"
    dft_us = step_kernels["band_dft"]["avg_us"]
    # algorithmic flops of the band DFT: 2 flops x M rows x N samples x 2C real outputs (one product;
    # the kernel issues six split-FP16 products over 128-row tiles and 16-column-padded tiles, so
    # frac <= 1/6 by construction; issued_frac counts the tensor work it actually issues)
    dft_flops = 2.0 * M * N * (2 * C)
    bn_tiles = -(-2 * C // 160)
    bn = -(-(-(-2 * C // bn_tiles)) // 16) * 16
    issued = 6 * 2.0 * (-(-M // 128) * 128) * (-(-N // 64) * 64) * (bn_tiles * bn)
    f16_peak = peaks["bf16_tflops"]  # dense FP16 runs at the dense BF16 rate (same nominal figure)
    roofline = {"kernel": "band_dft", "bound": "tensor", "achieved": dft_flops / (dft_us * 1e-6) / 1e12,
                "peak": f16_peak, "unit": "TFLOP/s", "traffic": TRAFFIC["band_dft"],
                "peak_source": "measured bf16 burst %.1f TFLOP/s (FP16 operands; dense FP16 = BF16 rate)" % peaks["bf16_tflops"],
                "issued_products": 6, "issued_tflops": issued / (dft_us * 1e-6) / 1e12}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    roofline["issued_frac"] = roofline["issued_tflops"] / roofline["peak"]

    # the whole chain against HBM: algorithmic bytes per frame = the raw frame
    # read once + the band map written once + the decisions written
    chain_bytes = 4.0 * M * N + 4.0 * M * C + 1.0 * M * C
    roofline_chain = {
        "bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"], "bytes_per_frame": chain_bytes,
        "per_frame": {"achieved": chain_bytes * value / world / 1e9,
                      "frac": chain_bytes * value / world / 1e9 / peaks["hbm_gbs"]},
        "batched_8": {"achieved": chain_bytes * chain_batched["frames_per_s"] / 1e9,
                      "frac": chain_bytes * chain_batched["frames_per_s"] / 1e9 / peaks["hbm_gbs"]}}

    # end to end through the public API with host buffers: H2D frame, chain, D2H decisions
    host_x = [f.cpu().pin_memory() for f in frames[:4]]
    host_det = torch.empty((M, C), dtype=torch.uint8).pin_memory()
    xbuf = torch.empty((M, N), dtype=torch.float32, device="cuda")
    Pb = torch.empty((M, C), dtype=torch.float32, device="cuda")
    db = torch.empty((M, C), dtype=torch.uint8, device="cuda")

    def e2e_step(i):
        xbuf.copy_(host_x[i % 4], non_blocking=True)
        rc.rcfar_preprocess(h, xbuf, params, Pb)
        v = rc.rcfar_sat(h, Pb, value_bound=band.value_bound, mode=rc.RCFAR_SAT_TILE_I64)
        rc.rcfar_cfar(h, v, None, win, cut_lo, cut_hi, db)
        host_det.copy_(db, non_blocking=True)

    for i in range(3):
        e2e_step(i)
    torch.cuda.synchronize()
    e0.record()
    for i in range(args.steps):
        e2e_step(i)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist)
    e2e_per_call = {"value": world * args.steps / (e2e_ms / 1e3), "unit": "frames/s",
                    "path": "per-call loop on one stream: copy in, rcfar_preprocess, rcfar_sat, rcfar_cfar, copy out"}
    # end to end through the library's host-buffer entry point (the server):
    # every frame is submitted from pinned host memory and its decisions come
    # back to pinned host memory; copies and compute of different frames
    # overlap across the server's slots
    e2e = e2e_server(rc, torch, args, local, host_x, w, M, N, C, world, dist)
    e2e["per_call_loop"] = e2e_per_call

    # SAT + CFAR on the 8192 x 8192 square-law map
    sat_cfar = None
    if not args.no_map:
        R = 8192
        Pm = torch.from_numpy(synth.square_law_map(R, R, n_targets=200, seed=rank)).cuda()
        bound = float(Pm.max().item())
        detm = torch.empty((R, R), dtype=torch.uint8, device="cuda")
        wm = rc.make_window(16, 16, 4, 4, 1e-6)

        reps = 10

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            assert rc.rcfar_get_error(h) == rc.RCFAR_OK
            return e0.elapsed_time(e1) / reps

        # split path: exact int64 table S in HBM (reduce, carry scans,
        # downsweep), then the streaming table CFAR
        def satcfar():
            v = rc.rcfar_sat(h, Pm, value_bound=bound, mode=rc.RCFAR_SAT_I64)
            rc.rcfar_cfar(h, v, Pm, wm, 0, R - 1, detm)

        mms = timed(satcfar)
        rc.rcfar_trace_enable(h, True)
        for _ in range(reps):
            satcfar()
        tr = rc.rcfar_trace_read(h)
        rc.rcfar_trace_enable(h, False)
        cells = R * R
        sat_us = 1e3 * tr["sat"][1] / tr["sat"][0]
        cfar_us = 1e3 * tr["cfar"][1] / tr["cfar"][0]
        sat_bytes = cells * (4 + 8)       # read map fp32, write the table S int64
        cfar_bytes = cells * (8 + 4 + 1)  # read table and map (CUT values), write decisions
        dom, dom_us, dom_b = ("sat", sat_us, sat_bytes) if sat_us >= cfar_us else ("cfar", cfar_us, cfar_bytes)
        ach = dom_b / (dom_us * 1e-6) / 1e9
        split = {"value": cells / (mms * 1e-3) / 1e9, "unit": "Gcells/s", "ms": mms,
                 "kernels_us": {"sat": sat_us, "cfar": cfar_us}, "hbm_bytes_per_cell": 25,
                 "hbm_frac": (sat_bytes + cfar_bytes) / (mms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                 "roofline": {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                              "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                              "traffic": TRAFFIC.get("cfar_ring_8192" if dom == "cfar" else "sat_i64_8192")}}
        # fused path: one streaming kernel, the table never leaves shared memory
        detf = torch.empty_like(detm)

        def fused8():
            rc.rcfar_sat_cfar(h, Pm, bound, wm, 0, R - 1, detf)

        fms = timed(fused8)
        fused_bytes = cells * (4 + 1)  # read the map, write the decisions
        fach = fused_bytes / (fms * 1e-3) / 1e9
        fused = {"value": cells / (fms * 1e-3) / 1e9, "unit": "Gcells/s", "ms": fms, "hbm_bytes_per_cell": 5,
                 "decisions_identical_to_split": bool(torch.equal(detf, detm)),
                 "roofline": {"kernel": "sat_cfar_stream", "bound": "hbm", "achieved": fach,
                              "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": fach / peaks["hbm_gbs"],
                              "traffic": TRAFFIC.get("sat_cfar_stream_8192"),
                              "note": "bound on the SM side (shared-memory wavefronts and 64-bit integer issue), not on DRAM"}}
        best = fused if fms <= mms else split
        sat_cfar = {"value": best["value"], "unit": "Gcells/s", "ms": best["ms"],
                    "path": "fused" if best is fused else "split",
                    "hbm_frac": best["roofline"]["frac"] if best is fused else best["hbm_frac"],
                    "workload": "8192x8192 square-law map, 200 targets over 80 dB, training 16 / guard 4, Pfa 1e-6, "
                                "exact 64-bit fixed-point integral image, CUT values from the map",
                    "split": split, "fused": fused, "hbm_frac_split": split["hbm_frac"]}
        # greatest-of thresholds (16 lookups per CUT instead of 8) on both paths
        wg = rc.make_window(16, 16, 4, 4, 1e-6, kind=rc.RCFAR_CFAR_GO)

        def split_go():
            v = rc.rcfar_sat(h, Pm, value_bound=bound, mode=rc.RCFAR_SAT_I64)
            rc.rcfar_cfar(h, v, Pm, wg, 0, R - 1, detf)

        def fused_go():
            rc.rcfar_sat_cfar(h, Pm, bound, wg, 0, R - 1, detf)

        gs, gf = timed(split_go), timed(fused_go)
        sat_cfar["greatest_of"] = {"split_gcells_per_s": cells / (gs * 1e-3) / 1e9,
                                   "fused_gcells_per_s": cells / (gf * 1e-3) / 1e9}
        # the table's storage choices on the same map (precision study)
        sat_cfar["precision"] = precision_study(rc, torch, h, Pm, synth.map_case_window())

    latency = latency_small_frame(rc, torch, synth, local)

    batch = None
    if not args.no_batch:
        batch = batch_measure(rc, torch, synth, local, rank)

    serving = None
    if not args.no_serve:
        serving = serving_measure(rc, torch, synth, local, rank, args.serve_frames, args.serve_burst)
        if batch is not None and serving["time_compressed"]:
            for kind in ("host_memory", "device_memory"):
                tc = serving[kind]["time_compressed"]
                serving[kind]["sustained_vs_per_frame_path"] = tc["frames_per_s"] / batch["per_frame_path_frames_per_s"]
                if batch.get("per_frame_graph_frames_per_s"):
                    serving[kind]["sustained_vs_per_frame_graph"] = (tc["frames_per_s"] /
                                                                     batch["per_frame_graph_frames_per_s"])
            serving["sustained_vs_per_frame_path"] = serving["host_memory"]["sustained_vs_per_frame_path"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, n, el = oracle_rate()
        cpu = {"value": v, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} frames of 1024x4096 in {el:.1f} s, numpy FP64 (BLAS threads = all cores)",
               "single_core": oracle_rate_single_core()}

    rc.rcfar_destroy(h)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE,
            "data": "synthetic (seeded UWB radar frames shaped like the paper's)",
            "config": {"workload": "full chain, one 1024x4096 raw frame per step (8 targets, training 16, guard 4, "
                                   "Pfa 1e-6, mean filter 5, fs 20 Hz)",
                       "l2": "inputs larger than L2: ring of 16 distinct frames (268 MB)",
                       "parallelism": f"replicas x{world}"},
            "timing": timing, "roofline": roofline, "roofline_chain": roofline_chain,
            "sat_cfar_gcells_per_s": sat_cfar["value"] if sat_cfar else None,
            "sat_cfar_hbm_frac": sat_cfar["hbm_frac"] if sat_cfar else None,
            "latency_cfg1": latency,
            "kernels": step_kernels, "sat_cfar": sat_cfar, "batch": batch,
            "serving": serving, "variants": variants, "chain_batched": chain_batched, "chain_sat_cfar": chain_map,
            "e2e": e2e,
            "cpu_baseline": cpu, "clocks": clk, "gpu_launches": launches_per_step * args.steps,
            "peaks": peaks["source"]}
    print(json.dumps(line), flush=True)


def profile_case(args):
    """Small fixed workloads for ncu captures: each runs its kernels three times."""
    import torch
    import synth
    import paper_2012_11077_gb300 as rc
    torch.cuda.set_device(0)
    if args.profile == "map":
        n = args.map_size
        h = rc.rcfar_create(device=0, max_rows=n, max_cols=n, max_n=4096, max_window=40, max_frames=1,
                            batch_bytes=1 << 24)
        Pm = torch.from_numpy(synth.square_law_map(n, n, n_targets=200, seed=0)).cuda()
        det = torch.empty((n, n), dtype=torch.uint8, device="cuda")
        w = rc.make_window(16, 16, 4, 4, 1e-6)
        bound = float(Pm.max().item())
        for _ in range(3):
            v = rc.rcfar_sat(h, Pm, value_bound=bound, mode=rc.RCFAR_SAT_I64)
            rc.rcfar_cfar(h, v, Pm, w, 0, n - 1, det)
    elif args.profile == "fused":
        n = args.map_size
        h = rc.rcfar_create(device=0, max_rows=n, max_cols=n, max_n=4096, max_window=40, max_frames=1,
                            batch_bytes=1 << 24)
        Pm = torch.from_numpy(synth.square_law_map(n, n, n_targets=200, seed=0)).cuda()
        det = torch.empty((n, n), dtype=torch.uint8, device="cuda")
        w = rc.make_window(16, 16, 4, 4, 1e-6)
        bound = float(Pm.max().item())
        for _ in range(3):
            rc.rcfar_sat_cfar(h, Pm, bound, w, 0, n - 1, det)
    elif args.profile in ("chain", "os"):
        h = rc.rcfar_create(device=0, max_rows=1024, max_cols=512, max_n=4096, max_window=40, max_frames=1,
                            batch_bytes=1 << 24)
        case = synth.large_frame_case(0)
        x = torch.from_numpy(synth.radar_frame(case.spec)).cuda()
        params = rc.make_pre_params(20.0, halo_c=case.halo_c)
        band = rc.rcfar_band_plan(case.spec.N, params)
        P = torch.empty((case.spec.M, band.cols), device="cuda")
        det = torch.empty((case.spec.M, band.cols), dtype=torch.uint8, device="cuda")
        w = case.window
        kind = rc.RCFAR_CFAR_OS if args.profile == "os" else rc.RCFAR_CFAR_CA
        win = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa, kind=kind)
        for _ in range(3):
            rc.rcfar_preprocess(h, x, params, P)
            if kind == rc.RCFAR_CFAR_OS:
                rc.rcfar_cfar_direct(h, P, win, band.k_lo - band.c0, band.k_hi - band.c0, det)
            else:
                rc.rcfar_sat_cfar(h, P, band.value_bound, win, band.k_lo - band.c0, band.k_hi - band.c0, det,
                                  map_cut=False)
    else:
        h = rc.rcfar_create(device=0, max_rows=1024, max_cols=1024, max_n=4096, max_window=32, max_frames=64,
                            batch_bytes=3 << 30)
        params = rc.make_pre_params(synth.FS_HZ, mean_len=5, halo_c=-1)
        keep, descs = [], []
        for c in synth.mixed_batch_cases(64, seed=100):
            x = torch.from_numpy(synth.radar_frame(c.spec)).cuda()
            w = c.window
            b = rc.rcfar_band_plan(c.spec.N, rc.make_pre_params(synth.FS_HZ, mean_len=5, halo_c=w.train_c + w.guard_c))
            d = torch.empty((c.spec.M, b.cols), dtype=torch.uint8, device="cuda")
            keep += [x, d]
            descs.append(rc.frame_desc(x, rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa), d))
        # the schedule the autotuner picks for this batch (four K blocks per band-DFT CTA, streaming
        # SAT + CFAR), set directly so that no timing runs precede the captured launches
        rc.rcfar_set_batch_tuning(h, rc.make_batch_tuning(4, rc.RCFAR_SAT_FUSED))
        for _ in range(3):
            rc.rcfar_run_batch(h, descs, params)
    torch.cuda.synchronize()
    st = rc.rcfar_get_error(h)
    rc.rcfar_destroy(h)
    print("profile case", args.profile, "status", st)
    return 0 if st == rc.RCFAR_OK else 1


def main():
    args = parse_args()
    if args.profile:
        sys.exit(profile_case(args))
    rank, world, local, dist = dist_setup()
    if args.impl == "reference":
        reference_arm(args, rank)
    else:
        ours(args, rank, world, local, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
