"""Host-side check of the band DFT's operand split (no GPU).

The tensor cores take FP16 operands and accumulate in FP32, rounding the
accumulator's adds toward zero. In each K block of 256 samples y is scaled by
a power of two so that its largest magnitude lies in [64, 128) and split into
the integer Y0 = rint(y 2^s) and the FP16 head Rh and tail Rt of the
remainder; the twiddles are scaled by 2^9 and split into the integer
T0 = rint(W 2^9) and the FP16 head T1 and tail T2 of the remainder. The
kernel accumulates ACC_A = sum Y0 T0 (integers below 2^24 in magnitude: exact
in FP32) and ACC_B = sum Y0 T1 + Y0 T2 + Rh T0 + Rh T1 + Rt T0 (inexact,
2^-8 of ACC_A's size).

Emulated in numpy on rows of the 1024 x 4096 frame, with ACC_B rounded toward
zero after every 16-sample MMA step:
  * the exactness precondition holds (|Y0| <= 128, |T0| <= 512, every ACC_A
    partial below 2^24);
  * the band bins stay within 1e-4 of FP64, relative to
    max(|bin|, 1e-6 x the map's largest bin), with room to spare;
  * the earlier split (FP16 head and tail of both operands, three products in
    one accumulator) under the same rounding model does not -- which is why
    the kernel splits as it does.
"""
import numpy as np

import oracle
import synth


def rz32(v):
    """Round to FP32 toward zero."""
    f = v.astype(np.float32)
    over = np.abs(f.astype(np.float64)) > np.abs(v)
    return np.where(over, np.nextafter(f, np.float32(0)), f).astype(np.float64)


def f16(x):
    return x.astype(np.float16).astype(np.float64)


def frame_rows():
    case = synth.large_frame_case(0)
    X = synth.radar_frame(case.spec).astype(np.float64)
    N = X.shape[1]
    P_o, band = oracle.preprocess_frame(X, synth.FS_HZ, case.mean_len, halo=case.halo_c)
    Y = oracle.preprocess.normalise(oracle.preprocess.mean_filter_slow_time(
        oracle.preprocess.detrend_fast_time(X), case.mean_len))
    rows = np.array([845, 282, 284] + list(range(0, X.shape[0], 32)))  # target rows and a spread
    c = Y[rows].mean(axis=1, keepdims=True)
    k = np.arange(band.c0, band.c1 + 1)
    ph = 2.0 * np.pi * ((k[:, None] * np.arange(N)[None, :]) % N) / N
    W = np.concatenate([np.cos(ph), -np.sin(ph)])  # [2C][N]
    return Y[rows] - c, c, W, k, N, P_o[rows], np.abs(P_o).max()


def magnitude(out, c, k, N):
    C = len(k)
    return np.hypot(out[:, :C] + N * c * (k == 0), out[:, C:])


def floored_rel_err(g, o, omax):
    return np.abs(g - o) / np.maximum(np.abs(o), 1e-6 * omax)


def exact_split_dft(yd, W):
    R, N = yd.shape
    T0 = np.rint(W * 512.0)
    T1 = f16(W * 512.0 - T0)
    T2 = f16(W * 512.0 - T0 - T1)
    assert np.abs(T0).max() <= 512
    out = np.zeros((R, W.shape[0]))
    for b0 in range(0, N, 256):
        sl = slice(b0, b0 + 256)
        mx = np.abs(yd[:, sl]).max(axis=1, keepdims=True)
        s = 7 - np.frexp(np.where(mx > 0, mx, 1.0))[1]
        v = yd[:, sl] * 2.0 ** s
        assert np.all(np.abs(v) < 128)
        Y0 = np.rint(v)
        Rh = f16(v - Y0)
        Rt = f16(v - Y0 - Rh)
        accA = np.zeros_like(out)
        accB = np.zeros_like(out)
        for k0 in range(0, min(256, N - b0), 16):
            ks, kg = slice(k0, k0 + 16), slice(b0 + k0, b0 + k0 + 16)
            accA += Y0[:, ks] @ T0[:, kg].T
            assert np.abs(accA).max() <= 2.0 ** 24
            for A, B in ((Y0, T2), (Y0, T1), (Rh, T0), (Rh, T1), (Rt, T0)):
                accB = rz32(accB + A[:, ks] @ B[:, kg].T)
        part = (accA.astype(np.float32) + accB.astype(np.float32)).astype(np.float64)
        out += part * 2.0 ** (-s - 9)
    return out


def head_tail_dft(yd, W):
    R, N = yd.shape
    wh = f16(W)
    wt = f16(W - wh)
    out = np.zeros((R, W.shape[0]))
    for b0 in range(0, N, 256):
        sl = slice(b0, b0 + 256)
        mx = np.abs(yd[:, sl]).max(axis=1, keepdims=True)
        s = 14 - np.frexp(np.where(mx > 0, mx, 1.0))[1]
        v = yd[:, sl] * 2.0 ** s
        yh = f16(v)
        yt = f16(v - yh)
        acc = np.zeros_like(out)
        for k0 in range(0, min(256, N - b0), 16):
            ks, kg = slice(k0, k0 + 16), slice(b0 + k0, b0 + k0 + 16)
            for A, B in ((yt, wh), (yh, wt), (yh, wh)):
                acc = rz32(acc + A[:, ks] @ B[:, kg].T)
        out += acc * 2.0 ** -s
    return out


def test_exact_head_split_holds_the_band_bins_and_the_old_split_does_not():
    yd, c, W, k, N, P_o, omax = frame_rows()
    # FP64 transform of the same y: the split's error alone
    new = floored_rel_err(magnitude(exact_split_dft(yd, W), c, k, N), P_o, omax)
    old = floored_rel_err(magnitude(head_tail_dft(yd, W), c, k, N), P_o, omax)
    assert new.max() < 1e-5, new.max()
    assert old.max() > 1e-4, old.max()
