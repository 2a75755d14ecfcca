"""The C-ABI library builds for sm_103a and exports every entry point declared in include/pump.h
(no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest

from paper_1607_06886_gb300 import build, pump

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pump.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pump_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("pump_build_graph", "pump_graph_build", "pump_plan", "pump_certify", "pump_explore", "pump_edge_masks",
              "pump_graph_from_csr", "pump_export", "pump_graph_destroy", "pump_status_str", "pump_set_allocator"):
        assert s in syms


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_status_strings_without_gpu():
    lib = pump.load()
    assert pump.status_str(pump.OK) == "ok"
    assert "capacity" in pump.status_str(pump.ERR_CAPACITY)
    assert pump.status_str(99) == "unknown status"


def test_invalid_arguments_rejected_before_any_device_work():
    lib = pump.load()
    out = ctypes.c_void_p()
    # NULL pointers and bad sizes are refused on the host
    assert lib.pump_build_graph(None, 0, 0, None, 0, None, 0, None, None, None, ctypes.byref(out)) == pump.ERR_INVALID_ARG
    assert lib.pump_graph_build(None, 0, 0, None, 0, None, 0, None, None, None, ctypes.byref(out)) == pump.ERR_INVALID_ARG
    assert lib.pump_graph_from_csr(0, None, None, None, None, 32, 0, None, 0, None, ctypes.byref(out)) == pump.ERR_INVALID_ARG
    assert lib.pump_plan(None, None, None, 0, None, None) == pump.ERR_INVALID_ARG
    assert lib.pump_plan_collect(None, None, None) == pump.ERR_INVALID_ARG
    assert lib.pump_explore(None, None, 1.0, None, None) == pump.ERR_INVALID_ARG
    assert lib.pump_edge_masks(None, None) == pump.ERR_INVALID_ARG
    assert lib.pump_edge_masks_list(None, None, 0, None, None, None) == pump.ERR_INVALID_ARG
    n = ctypes.c_size_t()
    assert lib.pump_export(None, 0, None, 0, ctypes.byref(n)) == pump.ERR_INVALID_ARG
    lib.pump_graph_destroy(None)


def test_mlp_invalid_arguments_rejected_on_the_host():
    lib = pump.load()
    out = ctypes.c_void_p()
    dims = (ctypes.c_int32 * 3)(224, 250, 16)   # a width that is not a multiple of 16
    assert lib.pump_mlp_create(2, dims, 0, ctypes.byref(out)) == pump.ERR_INVALID_ARG
    assert lib.pump_mlp_create(0, dims, 0, ctypes.byref(out)) == pump.ERR_INVALID_ARG
    assert lib.pump_mlp_create(2, None, 0, ctypes.byref(out)) == pump.ERR_INVALID_ARG
    assert lib.pump_mlp_param_count(None) == -1
    assert lib.pump_mlp_forward(None, None, 0, None, None) == pump.ERR_INVALID_ARG
    assert lib.pump_mlp_train(None, 16, 1, 1e-3, 0.1, 0, None, None) == pump.ERR_INVALID_ARG
    assert lib.pump_mlp_propose(None, None, 0, 1, 0, 0.1, None, None) == pump.ERR_INVALID_ARG
    lib.pump_mlp_destroy(None)


def test_binding_constants_match_the_header():
    """The binding's status codes, plan flags, graph flags and export kinds carry the header's
    values (the binding restates them for ctypes)."""
    text = open(os.path.join(ROOT, "include", "pump.h")).read()
    defines = {m.group(1): int(m.group(2), 0) for m in re.finditer(r"#define\s+(PUMP_\w+)\s+(0x[0-9a-fA-F]+|\d+)", text)}
    enums = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(PUMP_\w+)\s*=\s*(\d+)", text)}
    vals = {**defines, **enums}
    pairs = {"OK": "PUMP_OK", "ERR_INVALID_ARG": "PUMP_ERR_INVALID_ARG", "ERR_OOM": "PUMP_ERR_OOM",
             "ERR_CUDA": "PUMP_ERR_CUDA", "ERR_CAPACITY": "PUMP_ERR_CAPACITY", "ERR_TIMEOUT": "PUMP_ERR_TIMEOUT",
             "ERR_INFEASIBLE": "PUMP_ERR_INFEASIBLE", "NO_EARLY_STOP": "PUMP_NO_EARLY_STOP",
             "EXPLORE_ONLY": "PUMP_EXPLORE_ONLY", "STEPWISE": "PUMP_STEPWISE", "EXPLORE_GRID": "PUMP_EXPLORE_GRID",
             "NO_WAIT": "PUMP_NO_WAIT", "GRAPH_HSMC": "PUMP_GRAPH_HSMC", "GRAPH_SEPARATE_MASKS": "PUMP_GRAPH_SEPARATE_MASKS"}
    for py, c in pairs.items():
        assert c in vals, c
        assert getattr(pump, py) == vals[c], (py, getattr(pump, py), vals[c])
    for what, code in pump.EXPORT.items():
        name = "PUMP_EXPORT_" + what.upper()
        assert vals.get(name) == code, (name, vals.get(name), code)
