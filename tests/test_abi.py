"""Host-side checks of the C ABI: libpm.so builds, loads and exports every
symbol include/pm.h declares; configuration validation happens before any
CUDA call.  No compute call is made (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pm():
    from paper_2607_17929_gb300 import build
    build.build()
    from paper_2607_17929_gb300 import pm as m
    return m


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "pm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["pm_init", "pm_set_particles", "pm_project", "pm_solve", "pm_update", "pm_step",
                     "pm_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(pm):
    lib = C.CDLL(pm._SO)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_the_abi(pm):
    assert sorted(pm.EXPORTED) == declared_symbols()
    for s in declared_symbols():
        assert callable(getattr(pm, s))


def test_config_struct_layout(pm):
    assert C.sizeof(pm.pm_config) == 64
    assert pm.pm_config.stream.offset == 56


@pytest.mark.parametrize("n", [0, 7, 12, 20, 40, 1536, 2048])
def test_unsupported_mesh_sizes_rejected_on_host(pm, n):
    cfg = pm.pm_config(n, 10, 1000, 100.0, 0.31, 100.0, 0.0, 0, 0, None)
    h = C.c_void_p()
    assert pm.lib.pm_init(C.byref(cfg), C.byref(h)) == pm.PM_ERR_UNSUPPORTED_SIZE
    assert h.value is None


@pytest.mark.parametrize("field,value", [("n_steps", 0), ("n_part", 0), ("box_mpch", -1.0), ("omega_m", 0.0),
                                         ("z_final", 200.0), ("precision", 7), ("flags", 8)])
def test_invalid_config_rejected_on_host(pm, field, value):
    cfg = pm.pm_config(32, 10, 1000, 100.0, 0.31, 100.0, 0.0, 0, 0, None)
    setattr(cfg, field, value)
    h = C.c_void_p()
    assert pm.lib.pm_init(C.byref(cfg), C.byref(h)) == pm.PM_ERR_INVALID_ARG


def test_null_arguments(pm):
    assert pm.lib.pm_init(None, None) == pm.PM_ERR_INVALID_ARG
    assert pm.lib.pm_step(None) == pm.PM_ERR_INVALID_ARG
    pm.lib.pm_destroy(None)


def test_noalloc_wrapper_rejects_bad_position_arrays_before_any_call(pm, monkeypatch):
    """The allocation-free P(k) reads 3 * n doubles at the pointer: a flat array, an FP32 array or a tensor
    on the CPU must be refused by the binding with ValueError, before the library is reached."""
    import numpy as np
    import torch

    calls = []

    class NoLib:
        def __getattr__(self, name):
            calls.append(name)
            raise AssertionError(f"library reached: {name}")

    monkeypatch.setattr(pm, "lib", NoLib())
    bad = [torch.zeros(300, dtype=torch.float64),            # flat (3N,)
           torch.zeros((100, 3), dtype=torch.float32),       # FP32 read as FP64
           torch.zeros((100, 4), dtype=torch.float64),       # wrong row width
           torch.zeros((100, 3), dtype=torch.float64),       # host tensor, not on the current device
           np.zeros(300), np.zeros((100, 3), dtype=np.float32)]
    for arr in bad:
        with pytest.raises(ValueError):
            pm.pm_power_spectrum_noalloc(arr, 32, 0.31, 8)
    assert calls == []
