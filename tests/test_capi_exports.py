"""The C-ABI library builds for sm_103a, loads, and exports every function include/*.h declares.

No compute call is made here (CPU only)."""
import ctypes
import glob
import os
import re

import numpy as np

from paper_2502_15253_gb300 import fitcore

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fit_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fit_model_create", "fit_model_eval", "fit_model_expected", "fit_batch"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = fitcore.load(build_if_missing=True)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_struct_layouts_match_header_sizes():
    # sizes of the ABI structs as laid out by the binding (natural alignment, x86-64 / aarch64)
    assert ctypes.sizeof(fitcore.fit_instance) == 24
    assert ctypes.sizeof(fitcore.fit_result) == 32
    assert ctypes.sizeof(fitcore.fit_batch_opts) == 64
    assert fitcore.RESULT_DTYPE.itemsize == 32


def test_default_opts_and_error_message_without_gpu():
    L = fitcore.load(build_if_missing=True)
    o = fitcore.fit_batch_default_opts()
    assert o.history == 32 and o.max_iter > 0 and o.edm_tol > 0
    # invalid arguments are rejected on the host before any device work
    rc = L.fit_model_create(None, None)
    assert rc == -1
    assert b"null" in L.fit_last_error()
    assert np.isfinite(o.f_noise_rel)


def test_event_set_rejects_unsorted_bins_on_the_host():
    """fit_mc_create validates the events before it touches the device."""
    import ctypes as C
    L = fitcore.load()
    e = np.array([2.0, 3.0, 4.0], np.float32)
    c = np.zeros(3, np.uint8)
    w = np.ones(3, np.float32)
    b = np.array([0, 2, 1], np.int32)
    Lc = np.array([1000.0])
    h = C.c_void_p()
    rc = L.fit_mc_create(0, 1, Lc.ctypes.data, 3, e.ctypes.data, c.ctypes.data, w.ctypes.data,
                         b.ctypes.data, 3, C.byref(h))
    assert rc != 0 and b"not sorted" in L.fit_last_error()
    b = np.array([0, 1, 1], np.int32)
    c[1] = 1   # core out of range
    rc = L.fit_mc_create(0, 1, Lc.ctypes.data, 3, e.ctypes.data, c.ctypes.data, w.ctypes.data,
                         b.ctypes.data, 3, C.byref(h))
    assert rc != 0


def _create_error(spec):
    """fit_model_create on a description the library must reject before touching the device."""
    import pytest
    with pytest.raises(fitcore.FitError) as e:
        fitcore.Model(spec)
    return str(e.value)


def test_model_options_are_validated_on_the_host():
    import copy
    from paper_2502_15253_gb300 import synth
    base = synth.make_model("c0")
    s = copy.deepcopy(base)
    s.remap = 7
    assert "remap_mode" in _create_error(s)
    s = copy.deepcopy(base)
    s.osc_mode = 5
    assert "osc_mode" in _create_error(s)
    # the 3+1 formula with a held sin^2 2th14 outside [0, 1)
    s = copy.deepcopy(synth.make_model("c1s"))
    s.osc_idx = s.osc_idx.copy()
    s.osc_val = s.osc_val.copy()
    s.osc_idx[4] = -1
    s.osc_val[4] = 1.5
    assert "2th14" in _create_error(s)


def test_fit_options_are_validated_before_any_model_or_device_access():
    """fit_batch checks its options first: a bad history, restart count, block size or
    stopping rule is INVALID_ARG with a message naming it, before the models are read (the
    model handle here is a placeholder that must never be dereferenced) or the device used."""
    L = fitcore.load()
    fake = (ctypes.c_void_p * 1)(ctypes.c_void_p(8))
    inst = np.zeros(1, fitcore.INSTANCE_DTYPE)
    buf = np.zeros(64)
    res = np.zeros(1, fitcore.RESULT_DTYPE)
    cases = [("history", 0, "history must be 1..32"), ("history", 33, "history must be 1..32"),
             ("restarts", 9, "restarts must be 0..8"), ("threads", 48, "threads must be"),
             ("threads", 100, "threads must be"), ("edm_tol", 0.0, "edm_tol / max_iter"),
             ("max_iter", -1, "edm_tol / max_iter")]
    for field, value, msg in cases:
        o = fitcore.fit_batch_default_opts()
        setattr(o, field, value)
        rc = L.fit_batch(fake, 1, inst.ctypes.data, 1, buf.ctypes.data, None, buf.ctypes.data,
                         res.ctypes.data, ctypes.byref(o), None)
        assert rc == -1, field
        assert msg in L.fit_last_error().decode(), (field, L.fit_last_error())
    assert L.fit_batch(None, 1, inst.ctypes.data, 1, buf.ctypes.data, None, buf.ctypes.data,
                       res.ctypes.data, None, None) == -1
    # no instances: nothing to do, and nothing is read
    o = fitcore.fit_batch_default_opts()
    assert L.fit_batch(fake, 1, inst.ctypes.data, 0, buf.ctypes.data, None, buf.ctypes.data,
                       res.ctypes.data, ctypes.byref(o), None) == 0
