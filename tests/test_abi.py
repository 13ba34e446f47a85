"""The C-ABI library builds for sm_103a and exports every symbol that
include/*.h declares (no GPU needed; no compute calls)."""
import ctypes

from paper_2108_04209_gb300 import _lib as L


def test_library_exports_all_declared_symbols():
    names = L.exported_symbols()
    assert "superdc_secular_batched" in names and "superdc_opts_default" in names
    lib = L.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_opts_default_and_status_strings():
    o = L.default_opts()
    assert o.tau == 1e-10 and o.stop_c == 8.0 and o.max_iter == 50 and o.tile_roots == 0 and o.sched == 0
    for code in range(7):
        s = L.lib().superdc_status_string(code).decode()
        assert s.startswith("SUPERDC_")


def test_argument_errors_are_synchronous():
    lib = L.lib()
    o = L.default_opts()
    out = L.Rank1Out()
    # negative sizes / bad rho are rejected before anything is enqueued
    assert lib.superdc_secular_batched(-1, None, 0, None, None, 1.0, ctypes.byref(o), ctypes.byref(out), None) == 1
    assert lib.superdc_secular_batched(1, None, 1, None, None, 0.0, ctypes.byref(o), ctypes.byref(out), None) == 1
    o.max_iter = 0
    assert lib.superdc_secular_batched(1, None, 1, None, None, 1.0, ctypes.byref(o), ctypes.byref(out), None) == 1
    assert lib.superdc_opts_default(None) == 1
