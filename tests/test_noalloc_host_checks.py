"""Host-side argument checks of the allocation-free evaluation (fit_model_eval_noalloc) that
need no GPU: the library's decision on where the call's memory lives, called with attribute
values as cudaPointerGetAttributes reports them. A model or a buffer on another device than
the current one is rejected before any launch (another GPU's memory is not readable there
without peer access)."""
import ctypes as C

import numpy as np
import pytest

from paper_2502_15253_gb300 import fitcore

HOST, DEVICE, MANAGED = 1, 2, 3      # cudaMemoryType values
INVALID_ARG = -1


def _check(model_dev, cur_dev, types, devices):
    L = fitcore.load(build_if_missing=True)
    f = L.fitcore_noalloc_check_devices
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    t = np.ascontiguousarray(types, np.int32)
    d = np.ascontiguousarray(devices, np.int32)
    return f(model_dev, cur_dev, len(t), t.ctypes.data_as(C.POINTER(C.c_int)),
             d.ctypes.data_as(C.POINTER(C.c_int)))


def test_buffers_on_the_current_device_pass():
    assert _check(0, 0, [DEVICE, DEVICE, MANAGED], [0, 0, -1]) == 0
    assert _check(3, 3, [DEVICE] * 6, [3] * 6) == 0


def test_model_of_another_device_is_rejected():
    assert _check(1, 0, [DEVICE, DEVICE], [0, 0]) == INVALID_ARG


def test_buffer_of_another_device_or_host_is_rejected():
    assert _check(0, 0, [DEVICE, DEVICE], [0, 1]) == INVALID_ARG
    assert _check(0, 0, [DEVICE, HOST], [0, -1]) == INVALID_ARG
    assert _check(0, 0, [0], [-1]) == INVALID_ARG          # unregistered host memory
