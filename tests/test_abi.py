"""The C ABI library loads and exports every entry point include/nqs.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

from helpers import ROOT, ensure_built


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nqs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nqs_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ["nqs_create", "nqs_set_params", "nqs_init_chains", "nqs_sweep", "nqs_local_energy",
              "nqs_logpsi_grad", "nqs_stats", "nqs_destroy", "nqs_batch_create", "nqs_batch_sweep",
              "nqs_batch_step", "nqs_batch_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(ensure_built())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_validates_lattice_before_touching_the_gpu():
    lib = ctypes.CDLL(ensure_built())
    import paper_2601_20782_b300 as p
    hd = p.HamDesc(0, 2, 1, 1.0, 0.0, 1.0, 0)        # Lx = 2 is rejected
    md = p.ModelDesc(0, 4, 0, None)
    out = ctypes.c_void_p()
    st = p._lib.nqs_create(ctypes.byref(out), ctypes.byref(md), ctypes.byref(hd), 0)
    assert st == p.NQS_EINVAL
    assert b"Lx >= 3" in p._lib.nqs_last_error(None)
    assert not out.value


def test_null_context_is_rejected():
    import paper_2601_20782_b300 as p
    ensure_built()
    assert p._lib.nqs_sweep(None, None, 0, 0, 0, 0, 0, None, None, None, None, None) == p.NQS_EINVAL


def test_packing_helpers_round_trip():
    import numpy as np
    from helpers import pack_np, unpack_np
    s = np.random.default_rng(0).choice([-1, 1], size=(7, 45)).astype(np.int8)
    np.testing.assert_array_equal(unpack_np(pack_np(s), 45), s)


def test_batch_create_validates_before_touching_the_gpu():
    lib = ctypes.CDLL(ensure_built())
    import paper_2601_20782_b300 as p
    out = ctypes.c_void_p()
    items = (p.BatchItem * 1)()
    assert lib.nqs_batch_create(ctypes.byref(out), items, 0, 4, 1, 0, None) == p.NQS_EINVAL    # no items
    assert lib.nqs_batch_create(ctypes.byref(out), items, 1, 4, 1, 0, None) == p.NQS_EINVAL    # null context
    assert lib.nqs_batch_create(ctypes.byref(out), items, 1, 0, 0, 0, None) == p.NQS_EINVAL    # no sweeps
    assert lib.nqs_batch_create(ctypes.byref(out), items, 1, 4, 5, 0, None) == p.NQS_EINVAL    # burn-in > sweeps
    assert out.value is None
