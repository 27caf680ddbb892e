"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/henry.h declares (no compute calls)."""
import ctypes

import pytest

from paper_2403_17018_gb300 import binding as hb
from paper_2403_17018_gb300 import build as hbuild


@pytest.fixture(scope="module")
def lib():
    hbuild.build()
    return hb.load()


def test_every_declared_symbol_is_exported(lib):
    names = hb.declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_default_config_matches_table_1(lib):
    cfg = hb.default_config()
    assert (cfg.rho0, cfg.rho1, cfg.mu, cfg.g) == (1000.0, 1024.99, 1e-3, 9.8)
    assert (cfg.D, cfg.K0, cfg.phi0) == (18.8571e-6, 1.020408e-9, 0.35)
    assert (cfg.nx0, cfg.ny0, cfg.nt0, cfg.T) == (32, 16, 24, 43200.0)


def test_error_strings_and_invalid_config(lib):
    assert lib.henry_strerror(-1) == b"invalid argument"
    cfg = hb.default_config(n_xi=4)
    h = ctypes.c_void_p()
    assert lib.henry_create_levels(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert b"n_xi" in lib.henry_last_error()
    cfg = hb.default_config(nx0=30, ny0=15)
    assert lib.henry_create_levels(ctypes.byref(cfg), ctypes.byref(h)) == -5


@pytest.mark.parametrize("kw", [
    {"field_model": 2}, {"field_model": 1, "n_xi": 6}, {"krylov_iters": -1},
    {"krylov_iters": 65}, {"jac_lag": -1}, {"mg_small_cells": 513}, {"mg_small_cells": -1},
    {"vcycles": 0}, {"nu1": -1}, {"precision": 2}, {"nlevels": 0}, {"krylov_iters": 1},
    {"adjoint_rtol": 0.0}, {"adjoint_rtol": 1e-2}, {"adjoint_rtol": float("nan")},
    {"res_rows": -1}, {"res_rows": 65}, {"discretisation": 2}, {"mg_tb_cells": -1},
    {"guess_extrapolation": 7}, {"guess_extrapolation": -1}, {"jac_keep": 2},
])
def test_config_validation_rejects_out_of_range_options(lib, kw):
    """henry_create_levels validates the whole config before touching the
    device, so these checks run without a GPU: every option outside its
    documented range is rejected as an invalid argument."""
    cfg = hb.default_config(**kw)
    h = ctypes.c_void_p()
    assert lib.henry_create_levels(ctypes.byref(cfg), ctypes.byref(h)) == -1, kw
    assert not h.value


def test_new_options_default_off(lib):
    cfg = hb.default_config()
    assert (cfg.field_model, cfg.krylov_iters, cfg.jac_lag) == (0, 0, 0)
    assert cfg.mg_small_cells == 512 and cfg.newton_atol == 1e-11
    assert cfg.adjoint_rtol == 1e-14


@pytest.mark.parametrize("name", ["henry_residual_jacobian", "henry_residual_jacobian_noalloc"])
def test_batches_beyond_the_grid_limit_are_rejected_before_any_work(lib, name):
    """B > HENRY_MAX_BATCH (65535, one grid row per sample) is an invalid
    argument, returned before any pointer is touched or kernel enqueued, so
    this runs without a GPU (the pointers below are never dereferenced)."""
    cfg = hb.default_config()
    fake = ctypes.c_void_p(0x1000)
    fn = getattr(lib, name)
    rc = fn(ctypes.byref(cfg), 2, 1, 1.0, 65536, fake, fake, fake, fake, fake, fake, fake, None, None)
    assert rc == -1
    assert b"65535" in lib.henry_last_error()
