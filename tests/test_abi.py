"""The C-ABI library builds, loads and exports every entry point of
include/prost.h; host-side argument checks work without a GPU."""

import ctypes as C

import numpy as np
import pytest

import paper_1302_2073_gb300 as pg


def test_library_exports_every_declared_symbol():
    L = pg.lib()
    names = pg.header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), f"libprost does not export {n}"


def test_binding_covers_every_declared_symbol():
    for n in pg.header_functions():
        assert callable(getattr(pg, n)), n


def test_version_and_error_strings():
    assert pg.prost_version() == 102
    assert pg.prost_strerror(pg.PROST_EBADFRAME) == "frame has a non-finite entry"
    assert pg.prost_strerror(12345) == "unknown error"


def _ok():
    return dict(width=64, height=48, channels=3, k=10, p=0.25, mu=0.0, delta=0.35, omega=5e-5,
                t_init=5e-3, t_min=1e-4, i_init=100, n_cg=5, in_scale=1 / 255, in_offset=0.5,
                frame_dtype="u8")


def test_state_bytes_of_valid_parameters():
    n = pg.prost_state_bytes(pg.make_params(**_ok()))
    assert n > 64 * 48 * 3 * 10 * 4  # at least the subspace


@pytest.mark.parametrize("bad", [
    dict(width=0), dict(channels=5), dict(k=0), dict(k=33), dict(p=0.0), dict(p=2.5),
    dict(delta=0.0), dict(p=1.0, mu=0.0), dict(mu=-1.0), dict(omega=1.5), dict(t_init=0.0),
    dict(t_min=-1.0), dict(i_init=0), dict(n_cg=-1), dict(n_cg=33), dict(frame_dtype=7),
    dict(u_dtype=7), dict(mask_from=2), dict(width=2, height=2, channels=1, k=5),
    dict(in_scale=float("nan")),
    # k above the single-launch forms: the passes form only, float32 storage only
    dict(k=17, form=1), dict(k=20, form=2), dict(k=32, u_dtype="bf16"),
    dict(k=10, form=3, u_dtype="bf16"),
    # the resident form serves the register form's k only
    dict(k=11, form=4), dict(k=16, form=4),
])
def test_parameter_validation(bad):
    prm = dict(_ok())
    prm.update(bad)
    with pytest.raises(pg.ProstError) as ei:
        pg.prost_state_bytes(pg.make_params(**prm))
    assert ei.value.code == pg.PROST_EINVAL


def test_form_field_takes_the_five_forms_only():
    for form in (pg.PROST_FORM_AUTO, pg.PROST_FORM_GRID, pg.PROST_FORM_CLUSTER, pg.PROST_FORM_PASSES,
                 pg.PROST_FORM_RESIDENT):
        p = pg.make_params(**dict(_ok(), k=min(_ok()["k"], 10)), form=form)
        assert pg.prost_state_bytes(p) > 0
    for k in (17, 32):
        for form in (pg.PROST_FORM_AUTO, pg.PROST_FORM_PASSES):
            assert pg.prost_state_bytes(pg.make_params(**dict(_ok(), k=k), form=form)) > 0
    for form in (-1, 5):
        p = pg.make_params(**_ok())
        p.form = form
        with pytest.raises(pg.ProstError):
            pg.prost_state_bytes(p)


def test_null_arguments_are_rejected():
    L = pg.lib()
    assert L.prost_init(None, None, None) == pg.PROST_EINVAL
    h = C.c_void_p()
    assert L.prost_init(None, None, C.byref(h)) == pg.PROST_EINVAL
    assert L.prost_step(None, None, 0, None, None) == pg.PROST_EINVAL
    assert L.prost_sync(None) == pg.PROST_EINVAL
    assert L.prost_get_stats(None, None) == pg.PROST_EINVAL
    assert L.prost_inject_barrier_skew(None, 1) == pg.PROST_EINVAL
    assert L.prost_inject_wait_timeout(None, 0, 1000) == pg.PROST_EINVAL
    assert L.prost_step_async(None, None, None, None) == pg.PROST_EINVAL
    assert L.prost_wait(None) == pg.PROST_EINVAL
    assert L.prost_pre_get_state(None, None, None) == pg.PROST_EINVAL
    assert L.prost_pre_set_state(None, None, 0) == pg.PROST_EINVAL
    assert L.prost_window_inject_wait_timeout(None, 1, 1000) == pg.PROST_EINVAL
    L.prost_destroy(None)


@pytest.mark.parametrize("args", [
    (100, 3, 4, 8),          # m not a multiple of the channels
    (100, 1, 0, 8),          # k < 1
    (100, 1, 17, 8),         # k > 16
    (100, 1, 4, 0),          # empty window
    (100, 1, 4, 129),        # n > 128
    ((1 << 30) + 1, 1, 4, 8),  # m > 2^30
])
def test_window_arguments_are_checked_on_the_host(args):
    with pytest.raises(pg.ProstError) as ei:
        pg.prost_window_init(*args)
    assert ei.value.code == pg.PROST_EINVAL


@pytest.mark.parametrize("p,omega", [(0.0, 0.5), (2.5, 0.5), (float("nan"), 0.5), (0.5, -0.1), (0.5, 1.5)])
def test_window_exponent_and_weight_are_checked_on_the_host(p, omega):
    with pytest.raises(pg.ProstError):
        pg.prost_window_init(100, 1, 4, 8, p, omega)


@pytest.mark.parametrize("args", [
    (0, 480, 3, 160, 120, "u8", 100),        # empty input
    (640, 480, 3, 0, 120, "u8", 100),        # empty output
    (640, 480, 5, 160, 120, "u8", 100),      # more than 4 channels
    (1 << 16, 1 << 15, 1, 160, 120, "u8", 100),  # input plane over 2^30 pixels
    (640, 480, 3, 160, 120, 7, 100),         # unknown frame type
    (640, 480, 3, 160, 120, "u8", 0),        # no initialisation phase
])
def test_pre_processing_arguments_are_checked_on_the_host(args):
    with pytest.raises(pg.ProstError) as ei:
        pg.prost_pre_init(*args)
    assert ei.value.code == pg.PROST_EINVAL


def test_batch_and_median_arguments_are_checked_on_the_host():
    with pytest.raises(pg.ProstError):
        pg.prost_batch_init([])
    # a batch runs the single-launch forms only: refused before any device call
    for bad in (dict(k=17), dict(k=32), dict(form=pg.PROST_FORM_PASSES)):
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_batch_init([pg.make_params(**_ok()), pg.make_params(**dict(_ok(), **bad))])
        assert ei.value.code == pg.PROST_EINVAL
    L = pg.lib()
    m = np.zeros(16, np.uint8)
    ptr = m.ctypes.data_as(C.c_void_p)
    assert L.prost_median3x3(ptr, ptr, 0, 4, 0, None) == pg.PROST_EINVAL
    assert L.prost_median3x3(ptr, ptr, 4, -1, 0, None) == pg.PROST_EINVAL
    assert L.prost_median3x3(None, ptr, 4, 4, 0, None) == pg.PROST_EINVAL
