"""Argument checks of the C ABI that need no GPU: every entry point rejects a missing context or
handle and out-of-range sizes with GFH_ERR_ARG before touching the device; the host planners
reject invalid grids."""
import ctypes

import pytest


def test_null_handles_are_rejected(built_lib):
    gfh = built_lib
    L = gfh.lib()
    E = gfh.GFH_ERR_ARG
    pk = gfh.PeaksC(None, None, None, 1)
    assert L.gfh_plan_set_coarse(None, 64, 64, 32) == E
    assert L.gfh_plan_execute_tiles(None, ctypes.byref(pk), None, 0, None) == E
    assert L.gfh_synth_peaks(None, 1, 0, 10, 0, 9, 1, 0, None, None, None, 0, None) == E
    assert L.gfh_synth_images(None, 1, 0, 1, 300, 0, 299, 1, None, None, None, None) == E
    assert L.gfh_peaks_to_images(None, ctypes.byref(pk), 300, 0, 299, None, None) == E
    out = ctypes.c_void_p()
    assert L.gfh_cnn_create(None, 4, 1, ctypes.byref(out)) == E
    assert L.gfh_cnn_destroy(None) == gfh.GFH_OK
    assert L.gfh_cnn_param_count(None) == -1
    assert L.gfh_cnn_get_params(None, None, None) == E
    assert L.gfh_cnn_set_params(None, None) == E
    assert L.gfh_cnn_forward(None, None, 1, None) == E
    loss = ctypes.c_float()
    assert L.gfh_cnn_gradients(None, None, None, 1, ctypes.byref(loss)) == E
    assert L.gfh_cnn_train_step(None, None, None, 1, 1e-3, 0.0, ctypes.byref(loss)) == E
    assert L.gfh_propose_tiles(None, None, 1, None, 32, -1.0, None, None, None) == E
    assert L.gfh_conv3x3(None, 0, 32, 32, 2, 1, 32, None, None, None, None, None, None, None) == E
    g = gfh.GridC()
    assert L.gfh_select_squares(None, None, ctypes.byref(g), 5, 5, 3, None, None) == E
    assert L.gfh_coincide(None, None, 0, None, 0, 1.0, 1.0, 3.0, None, None) == E
    assert L.gfh_wait_check(None, 10) == E
    assert L.gfh_heterodyne(None, None, 10, 4096.0, 0.0, 300.0, 1e-12, 5.0, None) == E
    n = ctypes.c_int64()
    assert L.gfh_peakmap_complex(None, None, 4096, 1024.0, 2.0, 200, 300, 2.5, None, None, 0,
                                 ctypes.byref(n)) == E
    assert L.gfh_project_peaks(None, None, None, 0, 1.0, 2.0, 0.5, 0.0, 10, 20, None) == E


def test_grid_generators_reject_invalid_requests(built_lib):
    gfh = built_lib
    with pytest.raises(gfh.GfhError):
        gfh.n_grid(1.0, 3.0, 0.5, 100.0, 400.0, 1e-3, 100.0)      # n must exceed 1
    with pytest.raises(gfh.GfhError):
        gfh.n_grid(3.0, 2.0, 0.5, 100.0, 400.0, 1e-3, 100.0)      # n_hi < n_lo
    with pytest.raises(gfh.GfhError):
        gfh.k_segments(5.0, 0.5, 100.0, 400.0, 0.0, 1e-3)         # fdot_lo must be > 0
    with pytest.raises(gfh.GfhError):
        gfh.k_segments(5.0, 0.5, 100.0, 400.0, 1e-6, 1e-3, growth=0.5)
    with pytest.raises(gfh.GfhError) as e:
        gfh.k_segments(5.0, 0.5, 100.0, 400.0, 1e-9, 1e-3, growth=1.0, cap=10)
    assert e.value.code == gfh.GFH_ERR_SIZE                        # more segments than room
    assert gfh.n_grid(3.0, 3.0, 0.5, 100.0, 400.0, 1e-3, 100.0).tolist() == [3.0]
