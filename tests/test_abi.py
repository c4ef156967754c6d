"""The C-ABI library builds, loads and exports every symbol include/goat.h declares.

No compute call is made here (no GPU in the CPU suite)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"GOAT_API\s+[\w\s\*]*?\b(goat_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2111_05366_gb300 import _build
    try:
        return _build.build()
    except RuntimeError as e:  # no nvcc in this environment
        pytest.skip(str(e))


def test_header_declares_the_paper_calls():
    names = declared_symbols()
    for required in ["goat_match", "goat_gradient", "goat_sinkhorn", "goat_line_search", "goat_project"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_host_only_calls(lib_path):
    import paper_2111_05366_gb300 as goat
    assert goat.strerror(0) == "ok"
    assert "sm_103" in goat.strerror(goat.GOAT_ERR_UNSUPPORTED)
    p = goat.default_params()
    assert p.sk_max_iter == 500 and abs(p.sk_tol - 1e-3) < 1e-9 and p.sk_warm_start == 1
    assert p.direction == goat.GOAT_DIR_LOT
    assert set(goat.EXPORTED) == set(declared_symbols())


def test_direction_is_validated_before_any_device_work(lib_path):
    # an unknown direction, and FAQ in the batched path, are rejected by the argument
    # checks; the placeholder pointers are never dereferenced
    import ctypes

    import numpy as np

    import paper_2111_05366_gb300 as goat
    lib = goat.load()
    fake = ctypes.c_void_p(256)
    perm = np.zeros(8, dtype=np.int32)
    pp = perm.ctypes.data_as(ctypes.c_void_p)
    bad = goat.default_params(direction=7)
    assert lib.goat_match(fake, fake, 8, goat.GOAT_DTYPE_U8, None, ctypes.c_float(0.03), 1, ctypes.c_float(0.03),
                          ctypes.byref(bad), pp, None, None, None, ctypes.c_size_t(0), None) == goat.GOAT_ERR_INVALID_ARG
    faq = goat.default_params(direction=goat.GOAT_DIR_LAP)
    sizes = (ctypes.c_int * 1)(8)
    offs = (ctypes.c_longlong * 1)(0)
    assert lib.goat_match_batched(fake, fake, offs, sizes, 1, 1, ctypes.c_ulonglong(0), ctypes.c_float(0.03), 1,
                                  ctypes.c_float(0.03), ctypes.byref(faq), pp, None, None, None, None, None,
                                  ctypes.c_size_t(0), None) == goat.GOAT_ERR_INVALID_ARG


def test_binding_names_match_abi():
    import paper_2111_05366_gb300 as goat
    for name in ["goat_match", "goat_match_host", "goat_gradient", "goat_sinkhorn", "goat_line_search",
                 "goat_fw_update", "goat_project", "goat_objective"]:
        assert callable(getattr(goat, name))


def test_projection_schedule_defaults(lib_path):
    import paper_2111_05366_gb300 as goat
    o = goat.lap_options()
    assert o.max_rounds == 1 << 20 and o.head_rounds == 256
    assert o.tail_bids == -1 and o.tail_stall == -1 and o.sap_pops == -1
    assert o.head_stall == 16 and o.sap_every_phase == 0
    o = goat.lap_options(tail_bids=0, sap_pops=7)
    assert o.tail_bids == 0 and o.sap_pops == 7


def test_workspace_sizes_grow_with_the_form(lib_path):
    # host arithmetic only: the FP32 form doubles the operand buffers, the 8-bit
    # form adds four n x round_up(n, 128) byte operands
    import paper_2111_05366_gb300 as goat
    for n in (100, 1000, 4097):
        b16 = goat.workspace_bytes(n, goat.GOAT_DTYPE_U8, goat.GOAT_PREC_BF16)
        f32 = goat.workspace_bytes(n, goat.GOAT_DTYPE_U8, goat.GOAT_PREC_FP32)
        f8 = goat.workspace_bytes(n, goat.GOAT_DTYPE_U8, goat.GOAT_PREC_FP8)
        ld, ld8 = -(-n // 64) * 64, -(-n // 128) * 128
        assert f32 - b16 >= 2 * n * ld * 2 - 1024  # Xq and C1 gain a second BF16 term (256-byte rounding)
        assert f8 - b16 >= 4 * n * ld8 - 1024      # A8, B8, Q8, C8
        sp = goat.workspace_bytes(n, goat.GOAT_DTYPE_U8, goat.GOAT_PREC_BF16_SPLIT)
        sp8 = goat.workspace_bytes(n, goat.GOAT_DTYPE_U8, goat.GOAT_PREC_BF16_SPLIT8)
        assert sp8 - sp >= 2 * n * ld8 - 1024      # A8 and the lo term's C8
        assert goat.workspace_bytes(n, goat.GOAT_DTYPE_U8, goat.GOAT_PREC_BF16, host=True) > b16
