"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point
declared in include/*.h; argument checks that need no GPU reject bad input."""
import ctypes
import glob
import os
import re

import pytest

from paper_1908_10107_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"ORCA_API\s+[\w\s\*]*?\b(orca_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("orca_create", "orca_set_agents", "orca_step", "orca_get_state",
                     "orca_destroy", "orca_workspace_size", "orca_get_neighbors",
                     "orca_get_cells", "orca_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(abi.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert missing == []


def test_library_is_built_for_sm103a(lib):
    data = open(abi.LIB_PATH, "rb").read()
    assert b"sm_103a" in data or b"sm_103" in data


@pytest.mark.parametrize("bad", [
    dict(max_agents=0), dict(max_neighbors=0), dict(max_neighbors=33),
    dict(neighbor_dist=0.0), dict(neighbor_dist=-1.0), dict(dt=0.0), dict(cell_size=-1.0),
    dict(max_cells=-5),
])
def test_workspace_size_rejects_bad_params(lib, bad):
    kw = dict(max_agents=100, max_neighbors=10, neighbor_dist=10.0, dt=0.1)
    kw.update(bad)
    p = abi.make_params(**kw)
    with pytest.raises(abi.OrcaError) as e:
        abi.orca_workspace_size(p)
    assert e.value.status == abi.ORCA_ERR_ARG


def test_workspace_grows_with_capacity_and_recording(lib):
    small = abi.orca_workspace_size(abi.make_params(1000, 10, 10.0, 0.1))
    big = abi.orca_workspace_size(abi.make_params(100000, 10, 10.0, 0.1))
    rec = abi.orca_workspace_size(abi.make_params(1000, 10, 10.0, 0.1, flags=abi.ORCA_FLAG_RECORD))
    assert 0 < small < big and rec > small
    assert small % 256 == 0


def test_create_checks_arguments_before_touching_the_gpu(lib):
    p = abi.make_params(1000, 10, 10.0, 0.1)
    need = abi.orca_workspace_size(p)
    out = ctypes.c_void_p()
    # misaligned caller workspace
    assert lib.orca_create(ctypes.byref(p), ctypes.c_void_p(0x1001), need, ctypes.byref(out)) == abi.ORCA_ERR_ARG
    assert out.value is None
    assert "aligned" in lib.orca_last_error(None).decode()
    # too small
    assert lib.orca_create(ctypes.byref(p), ctypes.c_void_p(0x100000), need - 256,
                           ctypes.byref(out)) == abi.ORCA_ERR_NOMEM
    # null out / params
    assert lib.orca_create(ctypes.byref(p), None, 0, None) == abi.ORCA_ERR_ARG
    assert lib.orca_create(None, None, 0, ctypes.byref(out)) == abi.ORCA_ERR_ARG


def test_null_context_is_rejected(lib):
    assert lib.orca_step(None, 1, None) == abi.ORCA_ERR_ARG
    assert lib.orca_get_state(None, None, None, 0, None) == abi.ORCA_ERR_ARG
    assert lib.orca_destroy(None) == abi.ORCA_ERR_ARG
    m = ctypes.c_int32(-1)
    assert lib.orca_remove_arrived(None, ctypes.byref(m), None, 0, None) == abi.ORCA_ERR_ARG
    assert lib.orca_count_ops(None, 1) == abi.ORCA_ERR_ARG
    assert lib.orca_update_state(None, None, None, 0, None) == abi.ORCA_ERR_ARG
    assert lib.orca_step_host(None, None, None, 1, None, None, None) == abi.ORCA_ERR_ARG
    assert lib.orca_get_op_counters(None, None, None) == abi.ORCA_ERR_ARG


def test_status_strings(lib):
    assert abi.orca_status_string(abi.ORCA_OK) == "ok"
    assert abi.orca_status_string(abi.ORCA_ERR_NUMERIC) == "non-finite result"
    assert abi.orca_status_string(12345) == "unknown status"


def test_binding_refuses_to_run_without_library(tmp_path):
    with pytest.raises(abi.OrcaError):
        abi.load_library(str(tmp_path / "missing.so"))
