"""The C-ABI library builds, loads and exports every symbol include/cpb.h declares (no GPU)."""
import os
import re

import pytest

import paper_2206_07896_gb300 as cpb
from paper_2206_07896_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "cpb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cpb_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libs():
    cuda_build.build()
    return [cpb.lib(True), cpb.lib(False)]


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for must in ("cpb_stencil_launch", "cpb_heat_sum", "cpb_autotune", "cpb_status_string",
                 "cpb_version"):
        assert must in syms


def test_every_declared_symbol_is_exported(libs):
    for L in libs:
        for name in declared_symbols():
            assert hasattr(L._lib, name), f"{name} missing from {L.path}"


def test_binding_mirrors_the_header():
    assert set(declared_symbols()) == set(cpb.EXPORTED)
    for name in declared_symbols():
        assert callable(getattr(cpb, name))
        assert hasattr(cpb.Library, name)


def test_status_strings_and_version(libs):
    for L in libs:
        assert L.cpb_version() == 1
        assert L.cpb_status_string(cpb.CPB_ERR_SHARED_MEM) == "shared memory too small"
        assert L.cpb_status_string(99) == "unknown status"


def test_workspace_size_queries_need_no_gpu(libs):
    L = libs[0]
    assert L.cpb_heat_sum_workspace_bytes(0, 5) == 0
    assert L.cpb_heat_sum_workspace_bytes(8192, 8192) == 8 * 1024
    assert L.cpb_host_workspace_bytes(100, 10, cpb.CPB_F32) == 4 * 4096
