"""The Python binding rejects tensors the C ABI would misread, before any call
reaches the library (no GPU needed): a map that is not float32 (or float16
where the call takes it), decisions that are not uint8, thresholds that are
not float32, outputs smaller than the map, a status word that is not int32,
and tensors that are not on the current CUDA device."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rc():
    from paper_2012_11077_gb300 import build as b
    b.build()
    import paper_2012_11077_gb300 as pkg
    pkg.lib()
    return pkg


def _calls(rc, Pm, det, thr, status=None):
    w = rc.make_window(4, 4, 1, 1, 1e-3)
    return {
        "cfar_direct": lambda: rc.rcfar_cfar_direct(0, Pm, w, 0, 63, det, thr),
        "sat_cfar": lambda: rc.rcfar_sat_cfar(0, Pm, 10.0, w, 0, 63, det, thr),
        "sat_cfar_static": lambda: rc.rcfar_sat_cfar_static(Pm, 10.0, w, 0, 63, det, thr, status),
        "sat": lambda: rc.rcfar_sat(0, Pm, 10.0),
    }


def _good():
    return (torch.zeros((64, 64), dtype=torch.float32), torch.zeros((64, 64), dtype=torch.uint8),
            torch.zeros((64, 64), dtype=torch.float32))


@pytest.mark.parametrize("bad", ["map_f64", "map_i32", "det_i8", "det_small", "thr_f16", "thr_small", "det_1d"])
def test_bad_dtype_or_shape_raises_before_launch(rc, bad):
    Pm, det, thr = _good()
    if bad == "map_f64":
        Pm = Pm.double()
    elif bad == "map_i32":
        Pm = Pm.int()
    elif bad == "det_i8":
        det = det.to(torch.int8)
    elif bad == "det_small":
        det = det[:, :40]
    elif bad == "thr_f16":
        thr = thr.half()
    elif bad == "thr_small":
        thr = thr[:63]
    elif bad == "det_1d":
        det = det.reshape(-1)
    for name, call in _calls(rc, Pm, det, thr).items():
        if name == "sat" and not bad.startswith("map"):
            continue
        with pytest.raises(ValueError):
            call()


def test_status_word_must_be_int32(rc):
    Pm, det, thr = _good()
    with pytest.raises(ValueError):
        rc.rcfar_sat_cfar_static(Pm, 10.0, rc.make_window(4, 4, 1, 1, 1e-3), 0, 63, det, thr,
                                 torch.zeros((1,), dtype=torch.int64))


def test_host_tensors_are_not_device_buffers(rc):
    # the right dtypes and shapes, but in host memory: a device-pointer call must refuse them
    Pm, det, thr = _good()
    for call in _calls(rc, Pm, det, thr).values():
        with pytest.raises(ValueError, match="CUDA device"):
            call()


def test_preprocess_and_batch_outputs_checked(rc):
    p = rc.make_pre_params(20.0, halo_c=8)
    x = torch.zeros((32, 256), dtype=torch.float32)
    cols = rc.rcfar_band_plan(256, p).cols
    with pytest.raises(ValueError):  # map narrower than the band
        rc.rcfar_preprocess(0, x, p, torch.zeros((32, cols - 1), dtype=torch.float32))
    with pytest.raises(ValueError):  # float64 frame
        rc.rcfar_preprocess(0, x.double(), p, torch.zeros((32, cols), dtype=torch.float32))
    with pytest.raises(ValueError):  # decisions with fewer rows than the frame
        rc.frame_desc(x, rc.make_window(4, 4, 1, 1, 1e-3), torch.zeros((31, cols), dtype=torch.uint8))


def test_server_takes_host_tensors_of_the_right_type(rc):
    x = torch.zeros((32, 256), dtype=torch.float32)
    with pytest.raises(ValueError):
        rc.rcfar_server_submit(0, x.double(), rc.make_window(4, 4, 1, 1, 1e-3), torch.zeros((32, 40), dtype=torch.uint8),
                               tag=0)
    with pytest.raises(ValueError):
        rc.rcfar_server_submit(0, x, rc.make_window(4, 4, 1, 1, 1e-3), torch.zeros((32, 40), dtype=torch.float32),
                               tag=0)
