"""The C-ABI library loads and exports every entry point declared in
include/podecm.h; argument checks that need no GPU."""
import ctypes
import os
import re

import pytest

from paper_2307_16894_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "podecm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rom_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    return binding.lib()


def test_header_matches_binding():
    assert set(declared()) == set(binding.EXPORTED)


def test_exports(L):
    for f in declared():
        assert hasattr(L, f), f


def test_argument_errors_without_gpu(L):
    h = ctypes.c_void_p()
    assert L.rom_create(ctypes.byref(h), 5, 0, None) == binding.ROM_E_ARG
    assert not h.value
    assert L.rom_create(None, 2, 0, None) == binding.ROM_E_ARG
    assert L.rom_destroy(None) == binding.ROM_E_ARG
    assert L.rom_last_error(None) == b"null context"
    assert L.rom_step(None, None, None, None, None, None, None) == binding.ROM_E_ARG
    assert L.rom_state_destroy(None) == binding.ROM_E_ARG
    assert L.rom_set_geometry_aux(None, 1, None, None) == binding.ROM_E_ARG
    err = ctypes.create_string_buffer(256)
    assert L.rom_pod(None, 0, 1, None, None, None, None, None, 1, None, None, None, err, 256) == binding.ROM_E_ARG
    assert b"rom_pod" in err.value
    assert L.rom_ecm(None, 0, 10, None, None, 5, 0.0, 10.0, 5, None, None, None, None, None, err, 256) == binding.ROM_E_ARG
    assert b"rom_ecm" in err.value


def test_struct_layouts():
    assert ctypes.sizeof(binding.RomPhase) == 48
    assert ctypes.sizeof(binding.RomOpts) == 48   # 2 doubles, 7 int32, 4 bytes tail padding
    assert binding.RomOpts.fp64_residual.offset == 40
    assert binding.INFO_DTYPE.itemsize == 32
    # rom_aux_model: three int32, 4 bytes padding, six pointers
    assert ctypes.sizeof(binding.RomAuxModel) == 16 + 6 * 8 and binding.RomAuxModel.mu_ref.offset == 16
