"""CPU tests of the C ABI's argument checking: every entry point rejects
malformed arguments with PTN_ERR_INVALID_ARG (and the documented message)
before touching a device, and empty work returns PTN_OK.  No GPU needed."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from paper_2604_08467_gb300 import ptn

INVALID = 1


def _lib():
    return ptn.lib()


def test_null_handles_rejected():
    L = _lib()
    n = C.c_int64(0)
    assert L.ptn_contract_batch(None, None, 0, None, None, 0, 0, None, None, None) == INVALID
    assert L.ptn_sample_shots(None, None, None, None, None) == INVALID
    assert L.ptn_expval_grad(None, None, None, None, 0, None, None, None) == INVALID
    assert L.ptn_shots_merge(None, None, None) == INVALID
    assert L.ptn_plan_describe(None, 0, None, 0, None) == INVALID
    assert L.ptn_shots_info(None, C.byref(n), None, None, None, None, 0) == INVALID
    assert L.ptn_traj_info(None, C.byref(n), None, None, None, None, None) == INVALID
    assert b"NULL" in L.ptn_last_error() or b"is NULL" in L.ptn_last_error()


def test_batch_argument_checks():
    L = _lib()
    bo = ptn.ptn_batch_opts(2, 0, 0.0, 0.0)
    assert L.ptn_sample_shots_batch(None, 0, C.byref(bo), None, None, None) == 0      # empty batch
    assert L.ptn_sample_shots_batch(None, -1, C.byref(bo), None, None, None) == INVALID
    items = (ptn.ptn_batch_item * 1)()
    outs = (C.c_void_p * 1)()
    sts = (C.c_int * 1)()
    assert L.ptn_sample_shots_batch(items, 1, C.byref(bo), outs, sts, None) == INVALID   # NULL plan
    assert b"item 0" in L.ptn_last_error()


def test_sample_block_argument_checks():
    L = _lib()
    nc = C.c_int64(5)
    # block size out of range, no device work
    assert L.ptn_sample_block(None, 15, 0, None, None, None, 1, 0, 0, 0, None, None, None, 0, C.byref(nc), None) == INVALID
    # no parents: nothing to do, zero children
    assert L.ptn_sample_block(None, 4, 0, None, None, None, 0, 0, 0, 0, None, None, None, 0, C.byref(nc), None) == 0
    assert nc.value == 0
    assert L.ptn_allocate_shots(None, 0, 10, 0, 0, None, None) == INVALID


def test_plan_options_and_status_strings():
    L = _lib()
    for s, name in ptn.STATUS_NAMES.items():
        assert L.ptn_status_string(s).decode() == name
    circ = W.attach_noise(W.brickwork_1d(4, 2, np.random.default_rng(0)), [W.depolarizing_kraus(0.1)])
    plan = ptn.ptn_plan_path(circ, [4], hypersamples=2)
    d = plan.describe(detail=2)           # builds the gradient plan on the host
    assert d["expval"]["n_params"] == 0 and d["expval"]["pleaves"] == []


def test_header_is_plain_c():
    """include/ptn.h compiles as C99 (and C++17): the boundary uses no C++ types."""
    import os
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    header = os.path.join(root, "include", "ptn.h")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    r = subprocess.run([cc, "-fsyntax-only", "-x", "c", "-std=c99", "-Wall", "-Werror", header],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_plan_rejects_unknown_network_form():
    circ = W.attach_noise(W.brickwork_1d(4, 2, np.random.default_rng(0)), [W.depolarizing_kraus(0.1)])
    with pytest.raises(ptn.PtnError) as e:
        ptn.ptn_plan_path(circ, [4], hypersamples=2, network_form=3)
    assert e.value.status == INVALID


def test_tune_block_sizes_argument_checks():
    """Candidates outside 1..14, an empty list and probe sizes < 1 are refused
    before any device work."""
    rng = np.random.default_rng(42)
    circ = W.attach_noise(W.brickwork_1d(6, 3, rng), [W.depolarizing_kraus(0.05)])
    for cands, pt, ps in (([15], 4, 100), ([0, 2], 4, 100), ([2], 0, 100), ([2], 4, 0)):
        with pytest.raises(ptn.PtnError) as e:
            ptn.ptn_tune_block_sizes(circ, cands, probe_traj=pt, probe_shots=ps, stream=0)
        assert e.value.status == 1


def test_tune_tiles_argument_checks():
    lib = ptn.lib()
    assert lib.ptn_tune_tiles(None, None, 8, 2, None, None, None) == 1   # NULL handles
