"""FP64 preprocessing of the radar chain (paper Sec. II.A).

Test infrastructure: imported only by tests, the smoke check and the CPU
baseline of the benchmark. Never by the product path.

The paper lists the steps and delegates their parameters to its ref. [6]:
fast-time DC-shift removal and linear-trend subtraction; slow-time mean
filter, then normalisation; FFT of every slow-time signal; only the 0.3-0.8 Hz
respiration band is kept. Readings taken here where the paper is silent:
  * detrend: per trace (column n) least-squares line over the fast-time index m;
    subtracting the fitted line removes the DC shift as its intercept.
  * mean filter: centred moving average of odd length L along slow time,
    truncated at the ends with the divisor equal to the number of samples in
    range (constants are preserved).
  * normalisation: divide the whole frame by its maximum absolute value
    (unchanged if that maximum is 0).
  * transform: length-N DFT, rectangular window, no 1/N scaling, magnitude.
  * band: bins k_lo = ceil(f_lo N / fs) .. k_hi = floor(f_hi N / fs), both
    inclusive, evaluated in exact rational arithmetic; the stored map also
    carries `halo` bins each side (clipped to [0, floor(N/2)]) so that CFAR
    windows centred on band bins see the neighbouring spectrum.
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import NamedTuple

import numpy as np


class Band(NamedTuple):
    k_lo: int  # first respiration-band bin
    k_hi: int  # last respiration-band bin
    c0: int  # first stored bin (map column 0)
    c1: int  # last stored bin

    @property
    def cols(self) -> int:
        return self.c1 - self.c0 + 1


def band_plan(N: int, fs_hz: float, f_lo_hz: float = 0.3, f_hi_hz: float = 0.8, halo: int = 0) -> Band:
    """Respiration band bins of a length-N slow-time DFT (Sec. II.A, 0.3-0.8 Hz).

    Bin k has frequency k * fs / N. Inclusive band edges are computed with
    exact rationals from the decimal values of the frequencies.
    """
    fs = Fraction(str(fs_hz))
    lo = Fraction(str(f_lo_hz)) * N / fs
    hi = Fraction(str(f_hi_hz)) * N / fs
    k_lo = math.ceil(lo)
    k_hi = math.floor(hi)
    nyq = N // 2
    k_lo = max(k_lo, 0)
    k_hi = min(k_hi, nyq)
    c0 = max(0, k_lo - halo)
    c1 = min(nyq, k_hi + halo)
    return Band(k_lo, k_hi, c0, c1)


def detrend_fast_time(X: np.ndarray) -> np.ndarray:
    """DC-shift removal and linear-trend subtraction along fast time (Sec. II.A).

    For every trace n, fit x[m, n] ~ a_n + b_n * (m - mbar) by least squares over
    m = 0..M-1 and subtract the fit: a_n is the trace mean (the DC shift) and
    b_n = sum_m (m - mbar)(x - a_n) / sum_m (m - mbar)^2.
    """
    X = np.asarray(X, dtype=np.float64)
    M = X.shape[0]
    m = np.arange(M, dtype=np.float64) - (M - 1) / 2.0
    a = X.mean(axis=0)
    Xc = X - a[None, :]
    denom = float(m @ m)
    b = (m @ Xc) / denom if denom > 0 else np.zeros(X.shape[1])
    return Xc - np.outer(m, b)


def mean_filter_slow_time(Xp: np.ndarray, L: int) -> np.ndarray:
    """Centred moving average of odd length L along slow time (Sec. II.A).

    y[m, n] = (1 / |J_n|) * sum_{j in J_n} x'[m, j],  J_n = [n - h, n + h] cap [0, N),
    h = (L - 1) / 2.
    """
    if L < 1 or L % 2 == 0:
        raise ValueError("mean filter length must be odd and positive")
    Xp = np.asarray(Xp, dtype=np.float64)
    N = Xp.shape[1]
    h = (L - 1) // 2
    acc = np.zeros_like(Xp)
    cnt = np.zeros(N)
    for d in range(-h, h + 1):
        # contribution of sample n + d to output n, where n + d is in range
        lo = max(0, -d)
        hi = min(N, N - d)
        acc[:, lo:hi] += Xp[:, lo + d:hi + d]
        cnt[lo:hi] += 1.0
    return acc / cnt[None, :]


def normalise(Y: np.ndarray) -> np.ndarray:
    """Normalisation after the mean filter (Sec. II.A): divide by max |y| of the frame."""
    Y = np.asarray(Y, dtype=np.float64)
    mx = float(np.max(np.abs(Y))) if Y.size else 0.0
    return Y / mx if mx > 0 else Y.copy()


def normalise_row_zscore(Y: np.ndarray) -> np.ndarray:
    """Alternative reading of "then normalized" (Sec. II.A): each range bin's
    slow-time series scaled to zero mean and unit (population) standard
    deviation, z[m, n] = (y[m, n] - mean_n y[m, .]) / std_n y[m, .]; a
    constant row (std 0) becomes 0."""
    Y = np.asarray(Y, dtype=np.float64)
    mu = Y.mean(axis=1, keepdims=True)
    d = Y - mu
    sd = np.sqrt((d * d).mean(axis=1, keepdims=True))
    return np.where(sd > 0, d / np.where(sd > 0, sd, 1.0), 0.0)


def band_dft_magnitude(Y: np.ndarray, c0: int, c1: int) -> np.ndarray:
    """|DFT| of every slow-time signal at bins c0..c1 (Sec. II.A "FFT").

    P[m, j] = | sum_{n=0}^{N-1} y[m, n] exp(-2 pi i k n / N) |, k = c0 + j.
    The phase k*n is reduced modulo N in exact integer arithmetic before the
    FP64 exponential, so every twiddle is correctly computed for any N.
    """
    Y = np.asarray(Y, dtype=np.float64)
    N = Y.shape[1]
    k = np.arange(c0, c1 + 1, dtype=np.int64)
    n = np.arange(N, dtype=np.int64)
    t = np.outer(n, k) % N
    W = np.exp(-2j * np.pi * t / N)
    return np.abs(Y @ W)


def preprocess_frame(X: np.ndarray, fs_hz: float, mean_len: int = 5, halo: int = 0,
                     f_lo_hz: float = 0.3, f_hi_hz: float = 0.8, detector: str = "magnitude",
                     normalisation: str = "global_max"):
    """Whole Sec. II.A chain: raw X -> band-limited spectrum map P (FP64).

    detector: "magnitude" (|DFT|, the paper's "FFT" map) or "square" (|DFT|^2,
    the square-law map for which eq. 2's alpha is exact).
    normalisation: "global_max" (divide by the frame's max |y|) or
    "row_zscore" (normalise_row_zscore).
    Returns (P, band) with P of shape (M, band.cols).
    """
    if detector not in ("magnitude", "square") or normalisation not in ("global_max", "row_zscore"):
        raise ValueError("unknown detector or normalisation")
    X = np.asarray(X, dtype=np.float64)
    band = band_plan(X.shape[1], fs_hz, f_lo_hz, f_hi_hz, halo)
    Xp = detrend_fast_time(X)
    Y = mean_filter_slow_time(Xp, mean_len)
    Y = normalise(Y) if normalisation == "global_max" else normalise_row_zscore(Y)
    P = band_dft_magnitude(Y, band.c0, band.c1)
    if detector == "square":
        P = P * P
    return P, band
