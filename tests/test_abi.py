"""The C ABI library builds, loads and exports every function include/mci.h declares;
host-side argument validation (no GPU needed)."""
import ctypes

import numpy as np

import pytest

from paper_1802_10291_gb300 import mci


def test_exports_every_declared_symbol(mci_lib):
    declared = mci.header_functions()
    assert set(declared) == {"mci_plan", "mci_interp_1d", "mci_upsample_2d", "mci_upsample_2d_mirror", "mci_plan_info",
                             "mci_averaged_error", "mci_interp_1d_host",
                             "mci_destroy", "mci_error_string", "mci_interp_1d_noalloc",
                             "mci_corrector_num_params", "mci_corrector_create", "mci_corrector_forward",
                             "mci_corrector_loss_grad", "mci_corrector_train_step",
                             "mci_corrector_get_state", "mci_corrector_set_state", "mci_corrector_status",
                             "mci_corrector_destroy", "mci_generate_images", "mci_decimate", "mci_degrade",
                             "mci2_plan", "mci2_interp", "mci2_plan_info", "mci2_destroy",
                             "mci_debug_fail_allocation", "mci_tune_cache_save", "mci_tune_cache_load"}
    for name in declared:
        assert hasattr(mci_lib, name), name


def test_error_strings(mci_lib):
    for code in range(-7, 1):
        s = mci.error_string(code)
        assert s and s != "unknown status"
    assert mci.error_string(-99) == "unknown status"


def test_plan_bad_host_access(mci_lib):
    d = mci.make_desc([("identity",)], 16, 64, max_batch=4)
    d.host_access = 2
    h = ctypes.c_void_p()
    assert mci_lib.mci_plan(ctypes.byref(h), ctypes.byref(d), None) == mci.MCI_ERR_INVALID_ARG


@pytest.mark.parametrize("kw,status", [
    (dict(systems=[], P=16, T=64), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)] * 9, P=16, T=64), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=10, T=40), mci.MCI_ERR_UNSUPPORTED_SIZE),
    (dict(systems=[("identity",)], P=16, T=40), mci.MCI_ERR_UNSUPPORTED_SIZE),
    (dict(systems=[("identity",)], P=16384, T=16384), mci.MCI_ERR_UNSUPPORTED_SIZE),
    (dict(systems=[("identity",)], P=6, T=12), mci.MCI_ERR_UNSUPPORTED_SIZE),
    (dict(systems=[("identity",), ("hilbert",)], P=16, T=64, channels="fd"), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("deriv", 1)], P=16, T=64, channels="fd"), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=[16, 16], T=[64, 64]), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=16, T=64, max_batch=0), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=16, T=64, max_images=2, max_intermediate=100,
          outputs=("f", "hilbert")), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=16, T=64, max_images=2, max_intermediate=100,
          precision="fp64"), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",), ("deriv", 1)], P=16, T=64, channels="fd", complex_signal=True),
     mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=16, T=64, max_images=2, max_intermediate=100, complex_signal=True),
     mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=8192, T=8192, complex_signal=True), mci.MCI_ERR_UNSUPPORTED_SIZE),
    (dict(systems=[("identity",)], P=10, T=20, complex_signal=True), mci.MCI_ERR_UNSUPPORTED_SIZE),
    (dict(systems=[("identity",)], P=16, T=48, blur=(4, 1.0)), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=16, T=48, blur=(5, 0.0)), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=16, T=48, blur=(5, 1.0, -0.1)), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=16, T=48, blur=(257, 1.0)), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=16, T=48, blur=(-1, 1.0)), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[("identity",)], P=16, T=48, blur=(5, float("nan"))), mci.MCI_ERR_INVALID_ARG),
])
def test_plan_validation(mci_lib, kw, status):
    kw.setdefault("max_batch", 4)
    d = mci.make_desc(**kw)
    h = ctypes.c_void_p()
    assert mci_lib.mci_plan(ctypes.byref(h), ctypes.byref(d), None) == status
    assert h.value is None


def test_host_buffer_and_error_entry_points_check_arguments(mci_lib):
    assert mci_lib.mci_interp_1d_host(None, None, None, None, 1, None) == mci.MCI_ERR_INVALID_ARG
    assert mci_lib.mci_averaged_error(None, 0, None, 10, 1, None, None, None) == mci.MCI_ERR_INVALID_ARG


def test_null_arguments(mci_lib):
    assert mci_lib.mci_plan(None, None, None) == mci.MCI_ERR_INVALID_ARG
    assert mci_lib.mci_interp_1d(None, None, None, None, None, None, 1, None) == mci.MCI_ERR_INVALID_ARG
    assert mci_lib.mci_upsample_2d(None, None, None, None, None, None, None, None, 1, None) == \
        mci.MCI_ERR_INVALID_ARG
    assert mci_lib.mci_plan_info(None, None) == mci.MCI_ERR_INVALID_ARG
    assert mci_lib.mci_destroy(None) == mci.MCI_OK


def test_corrector_host_checks(mci_lib):
    from paper_1802_10291_gb300 import corrector
    from oracle import corrector as oc
    assert corrector.num_params() == oc.flatten(oc.unflatten(np.zeros(28353))).size == 28353
    assert mci_lib.mci_corrector_create(None, 16, None, None) == mci.MCI_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert mci_lib.mci_corrector_create(ctypes.byref(h), 0, None, None) == mci.MCI_ERR_INVALID_ARG
    assert mci_lib.mci_corrector_forward(None, None, None, 1, 8, 8, None) == mci.MCI_ERR_INVALID_ARG
    assert mci_lib.mci_corrector_destroy(None) == mci.MCI_OK
    assert mci_lib.mci_decimate(None, None, 1, 8, 8, 3, None) == mci.MCI_ERR_INVALID_ARG
    lib = corrector._lib()
    assert lib.mci_degrade(None, None, 1, 9, 9, 3, 5, 1.0, None) == mci.MCI_ERR_INVALID_ARG
    assert lib.mci_degrade(1 << 20, 1 << 21, 1, 9, 9, 3, 4, 1.0, None) == mci.MCI_ERR_INVALID_ARG
    assert lib.mci_degrade(1 << 20, 1 << 21, 1, 9, 9, 3, 5, -1.0, None) == mci.MCI_ERR_INVALID_ARG
    assert lib.mci_degrade(1 << 20, 1 << 21, 1, 8, 9, 3, 5, 1.0, None) == mci.MCI_ERR_INVALID_ARG
    assert mci_lib.mci_generate_images(None, None, 1, 8, 8, None) == mci.MCI_ERR_INVALID_ARG


def test_product_refuses_without_library(tmp_path):
    with pytest.raises(ImportError):
        mci._open(str(tmp_path / "missing.so"))


F2, DX2, DY2 = ("identity",), ("partial", 0, 1), ("partial", 1, 0)


@pytest.mark.parametrize("kw,status", [
    (dict(systems=[F2, DX2], grid=(1, 2), P=(16, 10), T=(32, 20)), mci.MCI_ERR_UNSUPPORTED_SIZE),
    (dict(systems=[F2, DX2], grid=(1, 2), P=(16, 2048), T=(32, 2048)), mci.MCI_ERR_UNSUPPORTED_SIZE),
    (dict(systems=[F2, DX2], grid=(1, 2), P=(16, 16), T=(24, 32)), mci.MCI_ERR_UNSUPPORTED_SIZE),
    (dict(systems=[F2, DX2], grid=(1, 2), P=(16, 16), T=(16 * 17, 32)), mci.MCI_ERR_UNSUPPORTED_SIZE),
    (dict(systems=[F2, DX2], grid=(0, 2), P=(16, 16), T=(32, 32)), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[F2] * 9, grid=(3, 3), P=(16, 16), T=(32, 32)), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[F2, ("riesz", 2)], grid=(1, 2), P=(16, 16), T=(32, 32)), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[F2, ("partial", -1, 0)], grid=(1, 2), P=(16, 16), T=(32, 32)), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[F2, DX2], grid=(1, 2), P=(16, 16), T=(32, 32), max_batch=0), mci.MCI_ERR_INVALID_ARG),
    (dict(systems=[F2, DX2], grid=(1, 2), P=(16, 16), T=(32, 32), max_batch=70000), mci.MCI_ERR_INVALID_ARG),
    # FP64, 8 channels of 1024 samples per column: the column pass needs more than 227 KB
    (dict(systems=[F2] * 8, grid=(2, 4), P=(1024, 1024), T=(2048, 2048), precision="fp64"),
     mci.MCI_ERR_UNSUPPORTED_SIZE),
])
def test_plan_2d_validation(mci_lib, kw, status):
    from paper_1802_10291_gb300 import mci2d
    kw.setdefault("max_batch", 2)
    systems = kw.pop("systems")
    d = mci2d.make_desc(systems, kw.pop("grid"), kw.pop("P"), kw.pop("T"), **kw)
    h = ctypes.c_void_p()
    assert mci2d._lib().mci2_plan(ctypes.byref(h), ctypes.byref(d), None) == status
    assert h.value is None


def test_2d_null_arguments(mci_lib):
    from paper_1802_10291_gb300 import mci2d
    lib = mci2d._lib()
    assert lib.mci2_plan(None, None, None) == mci.MCI_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.mci2_plan(ctypes.byref(h), None, None) == mci.MCI_ERR_INVALID_ARG
    assert lib.mci2_interp(None, None, None, 1, None) == mci.MCI_ERR_INVALID_ARG
    assert lib.mci2_plan_info(None, None, None, None) == mci.MCI_ERR_INVALID_ARG
    assert lib.mci2_destroy(None) == mci.MCI_OK


def test_tune_cache_json_round_trip(tmp_path):
    """The autotuner cache file: load merges a written object, save writes it back; malformed
    files and values outside 1 .. 64 are refused (host only, no device work)."""
    import json
    from paper_1802_10291_gb300 import mci
    src = tmp_path / "in.json"
    entries = {"generic-1d|fp32|real|P=768|T=2304|Min=1|Q=3|Test GPU|sm=4": 5,
               "generic-1d|fp64|complex|P=96|T=384|Min=2|Q=8|Test GPU|sm=4": 12}
    src.write_text(json.dumps(entries, indent=1))
    mci.mci_tune_cache_load(str(src))
    out = tmp_path / "out.json"
    mci.mci_tune_cache_save(str(out))
    saved = json.loads(out.read_text())
    for k, v in entries.items():
        assert saved[k] == v
    for bad in ('{"k": 0}', '{"k": 65}', '{"k" 3}', 'not json', '{"k": 3'):
        f = tmp_path / "bad.json"
        f.write_text(bad)
        with pytest.raises(mci.MciError) as e:
            mci.mci_tune_cache_load(str(f))
        assert e.value.status == mci.MCI_ERR_INVALID_ARG
    with pytest.raises(mci.MciError):
        mci.mci_tune_cache_load(str(tmp_path / "missing.json"))
