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
