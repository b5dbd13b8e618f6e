"""The C ABI without a GPU: the library loads, exports every function
include/tps.h declares, and rejects bad plan descriptors on the host."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2501_05938_gb300 import binding
from paper_2501_05938_gb300 import build as tps_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    tps_build.build()
    return binding.lib()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(tps_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"tps_plan", "tps_solve", "tps_solve_batched", "tps_solve_host_async"} <= names
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(binding.EXPORTS) <= names


def test_status_strings_and_version(lib):
    assert binding.version() >= 100
    assert binding.status_string(0) == "ok"
    assert "pivot" in binding.status_string(5)
    assert binding.status_string(99) == "unknown status"


@pytest.mark.parametrize("field,value", [("n_max", -1), ("dtype", 7), ("residency", 3), ("m", 1),
                                         ("m_reduced", 2), ("streams", 33), ("streams", -1),
                                         ("chunk", -5), ("reserved", 1), ("flags", 1 << 10),
                                         ("tol", -1.0), ("flags", 32)])
def test_plan_rejects_bad_descriptors_on_the_host(lib, field, value):
    d = binding.PlanDesc(n_max=1000, dtype=0)
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert lib.tps_plan(ctypes.byref(d), ctypes.byref(h)) == 1
    assert not h.value


@pytest.mark.parametrize("fields,status", [
    ({"flags": 128, "m": 101}, 1),                     # odd window
    ({"flags": 128, "m_reduced": 3}, 1),               # odd halo
    ({"flags": 128, "m": 1500, "m_reduced": 200}, 1),  # window + halos above 1792 rows
    ({"flags": 128, "m_reduced": -2}, 1),
    ({"flags": 128, "residency": 1}, 2),               # truncation is device-resident only
    ({"flags": 128, "dtype": 2}, 2),                   # and not for the refinement dtype
    ({"flags": 32 | 128, "residency": 1}, 2),
    ({"flags": 256}, 1),                               # overlap needs host residency
    ({"flags": 256 | 8, "residency": 1}, 2),           # and its own workspaces
    ({"flags": 256, "residency": 1, "dtype": 2}, 2),
])
def test_descriptor_flag_checks_on_the_host(lib, fields, status):
    d = binding.PlanDesc(n_max=1000, dtype=0)
    for k, v in fields.items():
        setattr(d, k, v)
    h = ctypes.c_void_p()
    assert lib.tps_plan(ctypes.byref(d), ctypes.byref(h)) == status
    assert not h.value


def test_flag_constants_match_the_header():
    hdr = open(os.path.join(ROOT, "include", "tps.h")).read()
    for name, val in (("TPS_GRAPH", binding.GRAPH), ("TPS_ZERO_COPY", binding.ZERO_COPY),
                      ("TPS_NO_ONCHIP", binding.NO_ONCHIP), ("TPS_TRUNCATE", binding.TRUNCATE),
                      ("TPS_TRACE", binding.TRACE), ("TPS_TUNE_PREDICT", binding.TUNE_PREDICT),
                      ("TPS_HOST_OVERLAP", binding.HOST_OVERLAP)):
        m = re.search(r"#define\s+" + name + r"\s+(\d+)u", hdr)
        assert m and int(m.group(1)) == val, name


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.tps_plan(None, ctypes.byref(h)) == 1
    assert lib.tps_plan_destroy(None) == 1
    assert lib.tps_solve(None, 10, None, None, None, None, None, None) == 1
    assert lib.tps_solve_host_async(None, 10, None, None, None, None, None, None) == 1
    assert lib.tps_solve_host_many_async(None, 2, 10, None, None, None, None, None, None) == 1
    assert lib.tps_plan_query(None, None) == 1
    sz = ctypes.c_size_t()
    assert lib.tps_workspace_size(None, ctypes.byref(sz)) == 1


def test_binding_checks_tensor_type_layout_and_length():
    # argument marshalling only: no plan, no library call is needed to reject these
    torch = pytest.importorskip("torch")
    plan = binding.Plan.__new__(binding.Plan)  # the checks use only the plan's dtype
    plan.dtype = "f64_df"
    good = [torch.zeros(10, dtype=torch.float64) for _ in range(5)]
    plan._arrays(10, *good)
    for bad in (torch.zeros(10, dtype=torch.float32), torch.zeros(20, dtype=torch.float64)[::2],
                torch.zeros(11, dtype=torch.float64)):
        with pytest.raises(binding.TpsError):
            plan._arrays(10, *good[:4], bad)
    plan.dtype = "f32"
    with pytest.raises(binding.TpsError):
        plan._arrays(10, *good)
    with pytest.raises(binding.TpsError):  # offsets the kernels read are int64
        binding.Plan._offsets(torch.zeros(3, dtype=torch.int32), None)
    keep, ptr = binding.Plan._offsets(torch.zeros(3, dtype=torch.int64), [0, 5, 10])
    assert keep.dtype == np.int64 and ptr.value == keep.ctypes.data
