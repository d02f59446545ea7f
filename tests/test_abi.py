"""The C-ABI library builds, loads and exports every entry point of
include/prost.h; host-side argument checks work without a GPU."""

import ctypes as C

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
    assert pg.prost_version() == 100
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
    dict(width=0), dict(channels=5), dict(k=0), dict(k=17), dict(p=0.0), dict(p=2.5),
    dict(delta=0.0), dict(p=1.0, mu=0.0), dict(mu=-1.0), dict(omega=1.5), dict(t_init=0.0),
    dict(t_min=-1.0), dict(i_init=0), dict(n_cg=-1), dict(n_cg=33), dict(frame_dtype=7),
    dict(u_dtype=7), dict(mask_from=2), dict(width=2, height=2, channels=1, k=5),
    dict(in_scale=float("nan")),
])
def test_parameter_validation(bad):
    prm = dict(_ok())
    prm.update(bad)
    with pytest.raises(pg.ProstError) as ei:
        pg.prost_state_bytes(pg.make_params(**prm))
    assert ei.value.code == pg.PROST_EINVAL


def test_reserved_field_must_be_zero():
    p = pg.make_params(**_ok())
    p.reserved = 1
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
    L.prost_destroy(None)
