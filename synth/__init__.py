"""Seeded synthetic inputs shaped like the paper's UWB radar frames.

This module holds only random-number draws and array assembly: it contains
none of the method's arithmetic (no detrending, filtering, transforms, tables
or thresholds). Both the CPU oracle tests and the GPU path take their inputs
from here, so the two sides always see the same bytes.

Frames follow the paper's data model (Sec. II.A): X in R^{M x N}, rows are
fast time (range bins), columns are slow time (traces). The paper's own frames
are 600 traces x 1024 samples (Sec. III); the sizes used here are the
workloads' sizes and every draw is seeded (numpy PCG64, platform independent).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

FS_HZ = 20.0  # slow-time sampling rate of every synthetic frame


@dataclasses.dataclass
class FrameSpec:
    """Recipe of one raw radar frame."""

    M: int  # fast-time samples (range bins)
    N: int  # slow-time samples (traces)
    n_targets: int = 2
    seed: int = 0
    fs_hz: float = FS_HZ
    noise_sigma: float = 0.1
    clutter_amp: float = 0.5
    n_clutter: int = 4
    target_sigma_bins: float = 3.0
    target_amp: float = 1.0
    f_lo_hz: float = 0.3
    f_hi_hz: float = 0.8


@dataclasses.dataclass
class FrameTruth:
    target_bins: np.ndarray  # range bin of each target
    target_freqs: np.ndarray  # respiration frequency of each target (Hz)
    clutter_bins: np.ndarray


def radar_frame(spec: FrameSpec, dtype=np.float32, return_truth: bool = False):
    """Raw frame X[M][N] (slow time contiguous).

    Draw order (fixed, one PCG64 stream seeded with spec.seed):
      1. per-range-bin DC offset o_m ~ U[-1, 1]              (M draws)
      2. per-trace linear fast-time drift slope s_n ~ U[-1e-3, 1e-3] (N draws)
      3. clutter bins: n_clutter distinct bins in [0, M)
      4. per target: bin m0 ~ U{0..M-1}, f ~ U[f_lo, f_hi], phase ~ U[0, 2pi)
      5. noise N(0, sigma^2)                                 (M*N draws)
    X[m, n] = o_m + s_n * m + clutter_amp * [m in clutter]
              + sum_t target_amp * exp(-(m - m0_t)^2 / (2 sigma_r^2))
                      * sin(2 pi f_t n / fs + phi_t)
              + noise[m, n]
    """
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    M, N = spec.M, spec.N
    offs = rng.uniform(-1.0, 1.0, size=M)
    drift = rng.uniform(-1e-3, 1e-3, size=N)
    clutter = rng.choice(M, size=min(spec.n_clutter, M), replace=False)
    m0 = np.empty(spec.n_targets, dtype=np.int64)
    freqs = np.empty(spec.n_targets)
    phases = np.empty(spec.n_targets)
    for t in range(spec.n_targets):
        m0[t] = rng.integers(0, M)
        freqs[t] = rng.uniform(spec.f_lo_hz, spec.f_hi_hz)
        phases[t] = rng.uniform(0.0, 2.0 * np.pi)
    noise = rng.normal(0.0, spec.noise_sigma, size=(M, N))

    m = np.arange(M, dtype=np.float64)[:, None]
    n = np.arange(N, dtype=np.float64)[None, :]
    X = noise
    X += offs[:, None]
    X += drift[None, :] * m
    X[clutter, :] += spec.clutter_amp
    for t in range(spec.n_targets):
        prof = spec.target_amp * np.exp(-((m - m0[t]) ** 2) / (2.0 * spec.target_sigma_bins ** 2))
        X += prof * np.sin(2.0 * np.pi * freqs[t] * n / spec.fs_hz + phases[t])
    X = np.ascontiguousarray(X.astype(dtype))
    if return_truth:
        return X, FrameTruth(m0, freqs, np.sort(clutter))
    return X


# --------------------------------------------------------------------------
# Workloads (sizes, windows and Pfa of the evaluated configurations)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Window:
    train_r: int
    train_c: int
    guard_r: int
    guard_c: int
    pfa: float


@dataclasses.dataclass
class ChainCase:
    """One raw frame plus its chain parameters."""

    spec: FrameSpec
    window: Window
    mean_len: int = 5

    @property
    def halo_c(self) -> int:
        return self.window.train_c + self.window.guard_c


def small_frame_case(seed: int = 0) -> ChainCase:
    """Single 256 x 512 frame, 2 targets, training 8, guard 2, Pfa 1e-4."""
    return ChainCase(FrameSpec(M=256, N=512, n_targets=2, seed=seed), Window(8, 8, 2, 2, 1e-4))


def large_frame_case(seed: int = 0) -> ChainCase:
    """Single 1024 x 4096 frame, 8 targets, training 16, guard 4, Pfa 1e-6."""
    return ChainCase(FrameSpec(M=1024, N=4096, n_targets=8, seed=seed), Window(16, 16, 4, 4, 1e-6))


TRAIN_SET = (4, 8, 16)
GUARD_SET = (1, 2, 4)
PFA_SET = (1e-3, 1e-4, 1e-6)


def mixed_batch_cases(n_frames: int = 64, seed: int = 0,
                      m_range=(128, 1024), n_range=(256, 4096)) -> List[ChainCase]:
    """Frames of uneven size with mixed windows.

    One PCG64 stream (seed) draws, per frame and in this order: M ~ U{m_lo..m_hi},
    N ~ U{n_lo..n_hi}, training ~ {4, 8, 16}, guard ~ {1, 2, 4},
    Pfa ~ {1e-3, 1e-4, 1e-6}, targets ~ U{0..10}, frame seed ~ U{0..2^31-1}.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_frames):
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        tr = int(rng.choice(TRAIN_SET))
        gd = int(rng.choice(GUARD_SET))
        pfa = float(rng.choice(PFA_SET))
        nt = int(rng.integers(0, 11))
        fseed = int(rng.integers(0, 2 ** 31 - 1))
        out.append(ChainCase(FrameSpec(M=M, N=N, n_targets=nt, seed=fseed), Window(tr, tr, gd, gd, pfa)))
    return out


@dataclasses.dataclass
class MapTargets:
    rows: np.ndarray
    cols: np.ndarray
    power: np.ndarray


def square_law_map(rows: int, cols: int, n_targets: int = 200, dyn_range_db: float = 80.0,
                   seed: int = 0, return_targets: bool = False):
    """CFAR input map: iid Exp(1) (square-law noise, mean 1) plus point targets.

    Draw order: noise Exp(1) (rows*cols), then per target row ~ U{0..rows-1},
    col ~ U{0..cols-1}, power = 10^(U[0, dyn_range_db]/10) added to that cell.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    P = rng.standard_exponential(size=(rows, cols), dtype=np.float64)
    tr = rng.integers(0, rows, size=n_targets)
    tc = rng.integers(0, cols, size=n_targets)
    pw = 10.0 ** (rng.uniform(0.0, dyn_range_db, size=n_targets) / 10.0)
    np.add.at(P, (tr, tc), pw)
    P = np.ascontiguousarray(P.astype(np.float32))
    if return_targets:
        return P, MapTargets(tr, tc, pw)
    return P


def map_case_window() -> Window:
    """Window used on the 8192 x 8192 square-law map: training 16, guard 4, Pfa 1e-6."""
    return Window(16, 16, 4, 4, 1e-6)


def integer_map(rows: int, cols: int, hi: int = 16, seed: int = 0) -> np.ndarray:
    """Small non-negative integer-valued map (exact in fp32 and fp64 sums)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, hi, size=(rows, cols)).astype(np.float32)


def serving_stream(n_requests: int = 10000, n_drones: int = 32, rate_hz: float = 200.0,
                   seed: int = 0, m_range=(128, 1024), n_range=(256, 4096), n_variants: int = 4):
    """Poisson request stream from simulated drones.

    Each drone is one radar: a fixed frame size M x N and a fixed window, drawn
    as in mixed_batch_cases; it has n_variants distinct frames (targets and
    noise differ). Requests arrive as a Poisson process of rate rate_hz; each
    comes from a uniformly drawn drone and carries one of its frames.
    One PCG64 stream (seed) draws, in this order: per drone M, N, training,
    guard, Pfa; per drone and variant the targets ~ U{0..10} and the frame
    seed; then the n_requests gaps ~ Exp(rate_hz), drones and variants.

    Returns (arrival_times_s, drone_ids, variants, drone_cases) with
    drone_cases[d][v] the ChainCase of drone d's frame v.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes = []
    for _ in range(n_drones):
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        tr = int(rng.choice(TRAIN_SET))
        gd = int(rng.choice(GUARD_SET))
        pfa = float(rng.choice(PFA_SET))
        shapes.append((M, N, Window(tr, tr, gd, gd, pfa)))
    drone_cases = []
    for M, N, w in shapes:
        vs = []
        for _ in range(n_variants):
            nt = int(rng.integers(0, 11))
            fseed = int(rng.integers(0, 2 ** 31 - 1))
            vs.append(ChainCase(FrameSpec(M=M, N=N, n_targets=nt, seed=fseed), w))
        drone_cases.append(vs)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    arrivals = np.cumsum(gaps)
    drones = rng.integers(0, n_drones, size=n_requests)
    variants = rng.integers(0, n_variants, size=n_requests)
    return arrivals, drones, variants, drone_cases
