"""The C ABI library on a machine without a GPU: it builds, loads, exports every
symbol the header declares, and its host-only helpers agree with the oracle."""
import math
import os
import re

import numpy as np
import pytest

import oracle
from oracle import cfar as ocfar

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rc():
    from paper_2012_11077_gb300 import build as b
    b.build()
    import paper_2012_11077_gb300 as pkg
    pkg.lib()
    return pkg


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "rcfar.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rcfar_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(rc):
    names = declared_symbols()
    assert len(names) >= 16
    L = rc.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(rc.EXPORTS) == names


def test_alpha_and_n_ref_match_oracle(rc):
    for tr, gd, pfa in [(8, 2, 1e-4), (16, 4, 1e-6), (4, 1, 1e-3), (1, 1, 1e-3), (12, 8, 1e-5)]:
        w = rc.make_window(tr, tr, gd, gd, pfa)
        nr = rc.rcfar_n_ref(w)
        assert nr == ocfar.n_ref(tr, tr, gd, gd)
        assert abs(rc.rcfar_alpha(nr, pfa) - ocfar.alpha(nr, pfa)) <= 1e-12 * ocfar.alpha(nr, pfa)
    w = rc.make_window(3, 5, 1, 2, 1e-3)
    assert rc.rcfar_n_ref(w) == ocfar.n_ref(3, 5, 1, 2)


def test_band_plan_matches_oracle(rc):
    for halo in (0, 5, 20):
        p = rc.make_pre_params(20.0, 0.3, 0.8, 5, halo)
        for N in list(range(5, 300)) + list(range(256, 4097, 7)) + [4000, 4096, 600]:
            o = oracle.band_plan(N, 20.0, 0.3, 0.8, halo)
            if o.cols < 1:  # nothing to store: rejected
                with pytest.raises(rc.RcfarError):
                    rc.rcfar_band_plan(N, p)
                continue
            b = rc.rcfar_band_plan(N, p)
            assert (b.k_lo, b.k_hi, b.c0, b.c1) == (o.k_lo, o.k_hi, o.c0, o.c1), N
            assert b.cols == o.cols and b.value_bound == N


def test_sat_scale_bounds_region_sums(rc):
    for bound, cells in [(1.0, 4096), (4096.0, 4096), (1e8, 1089), (3.0, 16641), (1e-20, 10)]:
        s = rc.rcfar_sat_scale(bound, cells)
        assert bound * cells * 2.0 ** s <= 2.0 ** 62
        assert bound * cells * 2.0 ** (s + 2) > 2.0 ** 62 or s == 100  # tight within 4x


def test_invalid_arguments_rejected_without_gpu(rc):
    with pytest.raises(rc.RcfarError) as e:
        rc.rcfar_alpha(0, 0.1)
    assert e.value.status == rc.RCFAR_ERR_INVALID_ARG
    with pytest.raises(rc.RcfarError):
        rc.rcfar_alpha(16, 1.0)
    with pytest.raises(rc.RcfarError):
        rc.rcfar_band_plan(0, rc.make_pre_params())
    with pytest.raises(rc.RcfarError) as e:
        rc.rcfar_create(max_rows=0)
    assert e.value.status == rc.RCFAR_ERR_INVALID_ARG
    with pytest.raises(rc.RcfarError):
        rc.rcfar_batch_bytes(10, 10, rc.make_pre_params(mean_len=4))
    assert rc.status_string(rc.RCFAR_ERR_RANGE).startswith("map value")


def test_batch_bytes_grows_with_frame(rc):
    p = rc.make_pre_params(20.0, 0.3, 0.8, 5, 20)
    a = rc.rcfar_batch_bytes(256, 512, p)
    b = rc.rcfar_batch_bytes(1024, 4096, p)
    assert 0 < a < b
    # at least the band map, its table and the statistics
    band = oracle.band_plan(4096, 20.0, halo=20)
    assert b >= 1024 * band.cols * 8 + 4096 * 8


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2012_11077_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_batch_tuning_argument_checks(rc):
    # invalid arguments are rejected before any device work
    import ctypes
    L = rc.lib()
    bad = rc.make_batch_tuning(-1)
    assert L.rcfar_set_batch_tuning(None, ctypes.byref(bad)) == rc.RCFAR_ERR_INVALID_ARG
    assert L.rcfar_get_batch_tuning(None, None) == rc.RCFAR_ERR_INVALID_ARG
    assert L.rcfar_tune_batch(None, None, 0, None, 1, None, None) == rc.RCFAR_ERR_INVALID_ARG


def test_threshold_factor_matches_oracle(rc):
    # the library's greatest-of / smallest-of factor (scaled term recurrence)
    # against the oracle's (log-gamma terms), and cell averaging's alpha / n_ref
    for tr, tc, gr, gc, pfa in [(16, 16, 4, 4, 1e-6), (4, 4, 1, 1, 1e-2), (2, 7, 0, 3, 1e-3), (1, 1, 1, 1, 0.1),
                                (32, 32, 8, 8, 1e-8), (1, 0, 0, 0, 0.25)]:
        for kind, okind in ((rc.RCFAR_CFAR_GO, ocfar.GO), (rc.RCFAR_CFAR_SO, ocfar.SO)):
            f, n = rc.rcfar_threshold_factor(rc.make_window(tr, tc, gr, gc, pfa, kind))
            assert n == ocfar.half_cells(tr, tc, gr, gc)
            o = ocfar.go_so_factor(okind, n, pfa)
            assert abs(f - o) <= 1e-12 * o, (kind, tr, tc, gr, gc, pfa, f, o)
        f, n = rc.rcfar_threshold_factor(rc.make_window(tr, tc, gr, gc, pfa))
        assert n == ocfar.n_ref(tr, tc, gr, gc)
        assert abs(f - ocfar.alpha(n, pfa) / n) <= 1e-14 * f


def test_window_kind_checks(rc):
    L = rc.lib()
    import ctypes
    f = ctypes.c_double()
    bad = [rc.make_window(4, 4, 1, 1, 1e-3, kind=4), rc.make_window(0, 2, 0, 1, 1e-3, kind=rc.RCFAR_CFAR_GO)]
    bad.append(rc.make_window(4, 4, 1, 1, 1e-3, os_rank=3))  # a rank for a non-OS window
    bad.append(rc.make_window(4, 4, 1, 1, 1e-3, kind=rc.RCFAR_CFAR_OS, os_rank=113))  # above n_ref = 112
    for w in bad:
        assert L.rcfar_threshold_factor(ctypes.byref(w), ctypes.byref(f), None) == rc.RCFAR_ERR_INVALID_ARG
    # the same columns-only window is valid for cell averaging (its training
    # cells all lie in the CUT's row, which neither half holds)
    ok = rc.make_window(0, 2, 0, 1, 1e-3)
    assert L.rcfar_threshold_factor(ctypes.byref(ok), ctypes.byref(f), None) == rc.RCFAR_OK


def test_os_factor_matches_oracle(rc):
    for tr, tc, gr, gc, pfa, k in [(4, 4, 1, 1, 1e-3, 0), (16, 16, 4, 4, 1e-6, 0), (1, 1, 0, 0, 1e-2, 0),
                                   (8, 8, 2, 2, 1e-4, 1), (8, 8, 2, 2, 1e-4, 416), (3, 5, 1, 2, 1e-2, 20)]:
        f, n = rc.rcfar_threshold_factor(rc.make_window(tr, tc, gr, gc, pfa, kind=rc.RCFAR_CFAR_OS, os_rank=k))
        assert n == ocfar.n_ref(tr, tc, gr, gc)
        kk = k or ocfar.os_rank_default(n)
        o = ocfar.os_factor(n, kk, pfa)
        assert abs(f - o) <= 1e-12 * o, (tr, tc, gr, gc, pfa, k, f, o)


def test_binding_structs_match_the_header(rc, tmp_path):
    # every ctypes structure of the binding has the size and field offsets the
    # C compiler gives the header's struct (a drift would corrupt arguments)
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [n for n in dir(rc) if n.startswith("rcfar_") and isinstance(getattr(rc, n), type)
               and issubclass(getattr(rc, n), ctypes.Structure)]
    assert len(structs) >= 10
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rcfar.h"', "int main(void) {"]
    for n in structs:
        lines.append(f'  printf("{n} size %zu\\n", sizeof({n}));')
        for f, _ in getattr(rc, n)._fields_:
            lines.append(f'  printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True, capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for n in structs:
        cls = getattr(rc, n)
        assert got[(n, "size")] == ctypes.sizeof(cls), n
        for f, _ in cls._fields_:
            assert got[(n, f)] == getattr(cls, f).offset, (n, f)


def test_static_entry_rejects_huge_windows_before_any_device_work(rc):
    # guard + train beyond what the CFAR's ring and strip can hold, including
    # half-widths whose int32 sum overflows, is refused on the host before any
    # CUDA call (the pointers below are never dereferenced)
    import ctypes
    L = rc.lib()
    fake = ctypes.c_void_p(16)
    for tr_r, tr_c, gd_r, gd_c in [(600_000_000, 0, 0, 0), (2**31 - 1, 1, 1, 1), (1, 2**31 - 1, 1, 1),
                                   (1025, 0, 0, 0), (0, 120, 0, 0), (0, 100, 0, 20)]:
        w = rc.make_window(tr_r, tr_c, gd_r, gd_c, 1e-3)
        st = L.rcfar_sat_cfar_static(fake, 64, 64, 64, ctypes.c_float(1.0), ctypes.byref(w), 0, 63, fake, 64,
                                     None, 0, None, None)
        assert st == rc.RCFAR_ERR_UNSUPPORTED, (tr_r, tr_c, gd_r, gd_c, st)
