"""The C-ABI library builds, loads and exports every symbol include/mdg.h declares; the
host-only entry points and the argument checks that run before any CUDA call work on a
machine without a GPU. CPU only (no compute call is made)."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import oracle
import paper_2606_08039_gb300 as mdg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mdg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mdg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(mdg_lib):
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(mdg_lib, s), f"{s} declared in mdg.h but not exported"
    # and the binding knows every one of them
    assert set(syms) <= set(mdg._SIGNATURES)


def test_constants_struct_layout(mdg_lib):
    assert mdg_lib.mdg_constants_size() == ctypes.sizeof(mdg.Constants)


def test_default_constants_match_paper_and_oracle(mdg_lib, golden_dir):
    c = mdg.Constants.cf2x().to_dict()
    g = json.load(open(os.path.join(golden_dir, "cf2x_paper_constants.json")))
    for k, v in g.items():
        if not k.startswith("_"):
            np.testing.assert_allclose(c[k], v["value"], rtol=1e-15, err_msg=k)
    # the oracle keeps its own table; both must agree on every field (printed or not)
    o = oracle.cf2x().to_dict()
    for k, v in o.items():
        np.testing.assert_allclose(c[k], v, rtol=1e-15, err_msg=k)


def test_hover_and_max_rpm(mdg_lib):
    c = mdg.Constants.cf2x()
    P = oracle.cf2x()
    assert c.hover_rpm() == pytest.approx(oracle.hover_rpm(P), rel=1e-15)
    assert c.max_rpm() == pytest.approx(oracle.max_rpm(P), rel=1e-15)
    assert mdg_lib.mdg_hover_rpm(None) < 0


def _create(n_envs, dpe, flags, c=None):
    h = ctypes.c_void_p()
    dpe = np.ascontiguousarray(dpe, dtype=np.int32)
    flags = np.ascontiguousarray(flags, dtype=np.uint32)
    rc = mdg.lib().mdg_create(n_envs, dpe.ctypes.data_as(ctypes.c_void_p), flags.ctypes.data_as(ctypes.c_void_p),
                              None if c is None else ctypes.byref(c), ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("n_envs,dpe,flags,needle", [
    (-1, [1], [0], "n_envs"),
    (2, [1, 2000], [0, 0], "drones_per_env"),
    (2, [1, -3], [0, 0], "drones_per_env"),
    (1, [4], [8], "unknown bits"),
])
def test_create_rejects_bad_arguments_before_any_cuda_call(mdg_lib, n_envs, dpe, flags, needle):
    rc, h = _create(n_envs, dpe, flags)
    assert rc == mdg.ERR_ARG and not h.value
    assert needle in mdg_lib.mdg_last_error().decode()


def test_create_rejects_bad_constants(mdg_lib):
    c = mdg.Constants.cf2x()
    c.mass = -1
    rc, _ = _create(1, [1], [0], c)
    assert rc == mdg.ERR_ARG
    c = mdg.Constants.cf2x()
    c.frame = 2
    rc, _ = _create(1, [1], [0], c)
    assert rc == mdg.ERR_ARG and "frame" in mdg_lib.mdg_last_error().decode()
    c = mdg.Constants.cf2x()
    c.integrator = 7
    rc, _ = _create(1, [1], [0], c)
    assert rc == mdg.ERR_ARG and "integrator" in mdg_lib.mdg_last_error().decode()
    c = mdg.Constants.cf2x()
    c.gnd_heights = -1
    rc, _ = _create(1, [1], [0], c)
    assert rc == mdg.ERR_ARG and "gnd_heights" in mdg_lib.mdg_last_error().decode()
    c = mdg.Constants.cf2x()
    c.controller = 5
    rc, _ = _create(1, [1], [0], c)
    assert rc == mdg.ERR_ARG and "controller" in mdg_lib.mdg_last_error().decode()
    c = mdg.Constants.cf2x().with_dsl()
    c.sp_rate_pos = 0.0
    rc, _ = _create(1, [1], [0], c)
    assert rc == mdg.ERR_ARG and "setpoint rates" in mdg_lib.mdg_last_error().decode()


@pytest.mark.parametrize("model", ["cf2x", "cf2p", "race"])
def test_model_constants_match_the_oracle(mdg_lib, model):
    """CF2P and RACE: the library's constants equal the oracle's own table field by field."""
    c = getattr(mdg.Constants, model)().to_dict()
    o = getattr(oracle, model)().to_dict()
    for k, v in o.items():
        np.testing.assert_allclose(c[k], v, rtol=1e-15, err_msg=k)


@pytest.mark.parametrize("model", ["cf2x", "cf2p", "race"])
def test_dsl_constants_match_the_oracle(mdg_lib, model):
    """mdg_controller_dsl and the oracle's own DSL tuning give the same gains, clamps and limits."""
    c = getattr(mdg.Constants, model)().with_dsl().to_dict()
    o = oracle.controller_dsl(getattr(oracle, model)()).to_dict()
    for k, v in o.items():
        np.testing.assert_allclose(c[k], v, rtol=1e-15, err_msg=k)
    assert c["controller"] == mdg.CTRL_DSL


def test_null_handle_calls_fail_cleanly(mdg_lib):
    L = mdg_lib
    assert L.mdg_step(None, None, None, 0, 5, None) == mdg.ERR_ARG
    assert L.mdg_step_obs(None, None, None, 0, 5, None, None, None, None) == mdg.ERR_ARG
    assert L.mdg_pid(None, None, None, None, None, None, None) == mdg.ERR_ARG
    assert L.mdg_obs(None, None, None, None, None, None) == mdg.ERR_ARG
    assert L.mdg_status(None, None, None, None) == mdg.ERR_ARG
    assert L.mdg_destroy(None) == mdg.OK
    assert L.mdg_num_drones(None) < 0
    assert L.mdg_create(0, None, None, None, None) == mdg.ERR_ARG


def test_sync_rejects_a_negative_limit_before_any_cuda_call(mdg_lib):
    assert mdg_lib.mdg_sync(None, -1) == mdg.ERR_ARG
    assert b"timeout_ms" in mdg_lib.mdg_last_error()


def test_noalloc_source_names_no_device_allocation():
    """mdg_step_obs_noalloc's translation unit calls no device allocator (comments and string
    literals aside): its only device memory is the static array and the caller's buffers."""

    src = open(os.path.join(ROOT, "paper_2606_08039_gb300", "csrc", "mdg_noalloc.cu")).read()
    code = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    code = re.sub(r"//[^\n]*", "", code)
    code = re.sub(r'"(\\.|[^"\\])*"', '""', code)
    banned = re.findall(r"\b(cudaMalloc\w*|cudaFree\w*|cuMemAlloc\w*|cuMemCreate|cudaMemPool\w*|"
                        r"cudaHostAlloc|cudaMallocHost)\b", code)
    assert banned == []
    assert "cudaGetSymbolAddress" in code and "cudaStreamIsCapturing" in code
