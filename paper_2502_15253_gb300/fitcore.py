"""Thin ctypes binding of the C ABI in include/fitcore.h (argument marshalling only).

Every computation runs in libfitcore.so. Arguments may be torch tensors (CPU or CUDA) or
numpy arrays; their data pointers are handed to the library, which stages host buffers
through device memory itself. If the library cannot be loaded this module raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class FitError(RuntimeError):
    pass


# ---- C structures (mirror include/fitcore.h) ----------------------------------------------
class fit_model_desc(C.Structure):
    _fields_ = [
        ("n_params", C.c_int),
        ("theta0", C.POINTER(C.c_double)), ("prior_sigma", C.POINTER(C.c_double)),
        ("scale", C.POINTER(C.c_double)),
        ("n_cov", C.c_int), ("cov_size", C.POINTER(C.c_int)), ("cov_idx", C.POINTER(C.c_int)),
        ("cov", C.POINTER(C.c_double)),
        ("osc_mode", C.c_int), ("osc_idx", C.c_int * 6), ("osc_val", C.c_double * 6),
        ("n_cores", C.c_int), ("core_power_idx", C.POINTER(C.c_int)),
        ("n_true", C.c_int), ("e_lo", C.c_double), ("e_hi", C.c_double),
        ("n_det", C.c_int), ("det_n_reco", C.POINTER(C.c_int)),
        ("det_response", C.POINTER(C.c_double)),
        ("n_ds", C.c_int), ("ds_det", C.POINTER(C.c_int)), ("ds_t", C.POINTER(C.c_double)),
        ("ds_baseline", C.POINTER(C.c_double)), ("ds_weight", C.POINTER(C.c_double)),
        ("ds_norm_idx", C.POINTER(C.c_int)), ("ds_eff_idx", C.POINTER(C.c_int)),
        ("ds_escale_idx", C.POINTER(C.c_int)), ("ds_shape_idx", C.POINTER(C.c_int)),
        ("n_bkg", C.c_int), ("bkg_ds", C.POINTER(C.c_int)),
        ("bkg_template", C.POINTER(C.c_double)), ("bkg_rate_idx", C.POINTER(C.c_int)),
        ("bkg_shape_idx", C.POINTER(C.c_int)),
        ("remap_mode", C.c_int),
    ]


class fit_model_info_t(C.Structure):
    _fields_ = [("n_params", C.c_int), ("n_data", C.c_int), ("n_datasets", C.c_int),
                ("n_true", C.c_int), ("device_bytes", C.c_size_t)]


class fit_instance(C.Structure):
    _fields_ = [("model", C.c_int), ("mask", C.c_uint32), ("data_off", C.c_int64),
                ("param_off", C.c_int64)]


class fit_batch_opts(C.Structure):
    _fields_ = [("edm_tol", C.c_double), ("max_iter", C.c_int), ("history", C.c_int),
                ("f_noise_rel", C.c_double), ("threads", C.c_int), ("blocks_per_sm", C.c_int),
                ("use_graph", C.c_int), ("time_budget_s", C.c_double), ("restarts", C.c_int),
                ("placement", C.c_int), ("engine", C.c_int), ("precondition", C.c_int)]


class fit_result(C.Structure):
    _fields_ = [("nll_min", C.c_double), ("edm", C.c_double), ("iters", C.c_int),
                ("n_evals", C.c_int), ("status", C.c_int), ("pad", C.c_int)]


RESULT_DTYPE = np.dtype([("nll_min", "<f8"), ("edm", "<f8"), ("iters", "<i4"),
                         ("n_evals", "<i4"), ("status", "<i4"), ("pad", "<i4")])
INSTANCE_DTYPE = np.dtype([("model", "<i4"), ("mask", "<u4"), ("data_off", "<i8"),
                           ("param_off", "<i8")])
assert RESULT_DTYPE.itemsize == C.sizeof(fit_result)
assert INSTANCE_DTYPE.itemsize == C.sizeof(fit_instance)

WS_MAX_TARGETS = 16
WS_MAX_MASKS = 8


class fit_warmstart_geom(C.Structure):
    _fields_ = [("slot0", C.c_int), ("onehot_slot", C.c_int), ("n_targets", C.c_int),
                ("target_idx", C.c_int * WS_MAX_TARGETS),
                ("target_scale", C.c_double * WS_MAX_TARGETS),
                ("n_uniform", C.c_int), ("uniform_idx", C.c_int * WS_MAX_TARGETS),
                ("uniform_half", C.c_double * WS_MAX_TARGETS),
                ("n_masks", C.c_int), ("masks", C.c_uint32 * WS_MAX_MASKS)]


STATUS = {0: "converged", 1: "maxiter", 2: "linesearch_fail", 3: "nonfinite",
          4: "mu_nonpositive", 5: "escale_nonmonotone", 6: "timeout", 7: "stalled"}

EXPORTS = ("fit_model_create", "fit_model_destroy", "fit_model_info", "fit_model_expected",
           "fit_model_eval", "fit_model_eval_noalloc", "fit_batch_default_opts", "fit_batch",
           "fit_tc_gemm", "fit_tc_gemm_status", "fit_last_error", "fit_kernel_launches",
           "fit_model_expected_tc", "fit_poisson_sample", "fit_mlp_create", "fit_mlp_destroy",
           "fit_mlp_forward", "fit_mlp_train_step", "fit_mlp_get_layer", "fit_mlp_set_layer",
           "fit_warmstart_features", "fit_warmstart_predict", "fit_warmstart_draw",
           "fit_warmstart_train", "fit_batch_autotune", "fit_batch_ex", "fit_profile_scan",
           "fit_wilks_interval", "fit_chi2_sf", "fit_mc_create", "fit_mc_destroy",
           "fit_mc_spectrum", "fit_mc_status", "fit_model_create_json", "fit_model_param_name",
           "fit_model_params", "fit_result_json", "fit_linear_start")


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libfitcore.so (building it first if asked). Raises FitError if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise FitError(f"libfitcore.so is not built ({_build.LIB}); run __graft_entry__.build()")
    L = C.CDLL(_build.LIB)
    vp = C.c_void_p
    L.fit_model_create.argtypes = [C.POINTER(fit_model_desc), C.POINTER(vp)]
    L.fit_model_destroy.argtypes = [vp]
    L.fit_model_info.argtypes = [vp, C.POINTER(fit_model_info_t)]
    L.fit_model_expected.argtypes = [vp, C.c_int, vp, vp, vp, vp]
    L.fit_model_eval.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp, vp]
    L.fit_model_eval_noalloc.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp, vp]
    L.fit_batch_default_opts.argtypes = [C.POINTER(fit_batch_opts)]
    L.fit_tc_gemm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, vp, C.c_int, C.c_int,
                              vp, C.c_int, vp, C.c_int, vp, vp, C.c_int, vp]
    L.fit_tc_gemm.restype = C.c_int
    L.fit_tc_gemm_status.restype = C.c_int
    L.fit_batch.argtypes = [C.POINTER(vp), C.c_int, vp, C.c_int, vp, vp, vp, vp,
                            C.POINTER(fit_batch_opts), vp]
    L.fit_model_expected_tc.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int, vp]
    L.fit_poisson_sample.argtypes = [C.c_int64, vp, C.c_uint64, C.c_uint64, vp, vp]
    L.fit_mlp_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(vp)]
    L.fit_mlp_destroy.argtypes = [vp]
    L.fit_mlp_destroy.restype = None
    L.fit_mlp_forward.argtypes = [vp, C.c_int, vp, vp, vp]
    L.fit_mlp_train_step.argtypes = [vp, C.c_int, vp, vp, C.c_float, C.c_float, vp, vp]
    L.fit_mlp_get_layer.argtypes = [vp, C.c_int, vp, vp, vp, vp]
    L.fit_mlp_set_layer.argtypes = [vp, C.c_int, vp, vp]
    L.fit_warmstart_features.argtypes = [vp, C.c_int, vp, vp, C.c_int, C.c_int, C.c_int, vp, vp]
    L.fit_warmstart_predict.argtypes = [vp, vp, C.c_int, vp, vp, C.c_int, C.c_int, C.c_int, vp,
                                        vp, vp, vp]
    L.fit_linear_start.argtypes = [vp, C.c_int, vp, vp, vp, vp]
    L.fit_linear_start.restype = C.c_int
    L.fit_warmstart_draw.argtypes = [vp, C.POINTER(fit_warmstart_geom), C.c_int, C.c_uint64,
                                     C.c_uint64, vp, vp, vp]
    L.fit_warmstart_train.argtypes = [vp, C.POINTER(vp), C.POINTER(fit_warmstart_geom), C.c_int,
                                      C.c_int, C.c_int, C.c_float, C.c_float, C.c_uint64, vp, vp]
    for f in ("fit_model_expected_tc", "fit_poisson_sample", "fit_mlp_create", "fit_mlp_forward",
              "fit_mlp_train_step", "fit_mlp_get_layer", "fit_mlp_set_layer",
              "fit_warmstart_features", "fit_warmstart_predict", "fit_warmstart_draw",
              "fit_warmstart_train"):
        getattr(L, f).restype = C.c_int
    L.fit_batch_autotune.argtypes = [C.POINTER(vp), C.c_int, vp, C.c_int, vp, vp, C.c_int,
                                     C.POINTER(fit_batch_opts), vp]
    L.fit_batch_autotune.restype = C.c_int
    L.fit_batch_ex.argtypes = [C.POINTER(vp), C.c_int, vp, C.c_int, vp, vp, vp, vp, vp,
                               C.POINTER(fit_batch_opts), vp]
    L.fit_batch_ex.restype = C.c_int
    L.fit_profile_scan.argtypes = [vp, vp, C.c_uint32, C.c_int, vp, C.c_int, vp, vp,
                                   C.POINTER(fit_batch_opts), vp, vp, vp, vp, vp, vp]
    L.fit_profile_scan.restype = C.c_int
    L.fit_wilks_interval.argtypes = [C.c_int, vp, vp, C.c_double, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]
    L.fit_wilks_interval.restype = C.c_int
    L.fit_chi2_sf.argtypes = [C.c_double, C.c_int]
    L.fit_chi2_sf.restype = C.c_double
    L.fit_mc_create.argtypes = [C.c_int, C.c_int, vp, C.c_int64, vp, vp, vp, vp, C.c_int,
                                C.POINTER(vp)]
    L.fit_mc_create.restype = C.c_int
    L.fit_mc_destroy.argtypes = [vp]
    L.fit_mc_destroy.restype = None
    L.fit_mc_spectrum.argtypes = [vp, C.c_int, vp, vp, vp]
    L.fit_mc_spectrum.restype = C.c_int
    L.fit_mc_status.argtypes = [vp]
    L.fit_mc_status.restype = C.c_int
    L.fit_model_create_json.argtypes = [C.c_char_p, C.POINTER(vp)]
    L.fit_model_create_json.restype = C.c_int
    L.fit_model_param_name.argtypes = [vp, C.c_int]
    L.fit_model_param_name.restype = C.c_char_p
    L.fit_model_params.argtypes = [vp, vp, vp]
    L.fit_model_params.restype = C.c_int
    L.fit_result_json.argtypes = [vp, vp, vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]
    L.fit_result_json.restype = C.c_int
    L.fit_last_error.restype = C.c_char_p
    L.fit_kernel_launches.restype = C.c_int64
    for f in ("fit_model_create", "fit_model_info", "fit_model_expected", "fit_model_eval",
              "fit_model_eval_noalloc", "fit_batch"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != 0:
        msg = load().fit_last_error().decode(errors="replace")
        raise FitError(f"{what} failed ({rc}): {msg}")


def _ptr(x):
    """Data pointer of a torch tensor / numpy array (must be contiguous), or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class Model:
    """A model resident on the current CUDA device (wraps fit_model*).

    Model(spec) builds it from a synth.ModelSpec through fit_model_create;
    Model.from_json(text) from a JSON configuration through fit_model_create_json."""

    def __init__(self, spec, _handle=None):
        L = load()
        self.spec = spec
        if _handle is not None:
            self._attach(_handle)
            return
        if getattr(spec, "map_priors", None):
            # priors on b = A theta exist only in the JSON schema (fit_model_create_json)
            h = C.c_void_p()
            _check(L.fit_model_create_json(spec.to_json().encode(), C.byref(h)),
                   "fit_model_create_json")
            self._attach(h)
            return
        keep = []

        def d(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data_as(C.POINTER(C.c_double))

        def i(a):
            a = np.ascontiguousarray(a, dtype=np.int32)
            keep.append(a)
            return a.ctypes.data_as(C.POINTER(C.c_int))

        s = spec
        m = fit_model_desc()
        m.n_params = s.n_params
        m.theta0, m.prior_sigma, m.scale = d(s.theta0), d(s.prior_sigma), d(s.scale)
        m.n_cov = len(s.cov_blocks)
        m.cov_size = i([len(ix) for ix, _ in s.cov_blocks] or [0])
        m.cov_idx = i(np.concatenate([ix for ix, _ in s.cov_blocks]) if s.cov_blocks else [0])
        m.cov = d(np.concatenate([c.ravel() for _, c in s.cov_blocks]) if s.cov_blocks else [0.0])
        m.osc_mode = s.osc_mode
        m.remap_mode = int(getattr(s, "remap", 0))
        for k in range(6):   # the 3+1 formula has six survival parameters, the others four
            m.osc_idx[k] = int(s.osc_idx[k]) if k < len(s.osc_idx) else -1
            m.osc_val[k] = float(s.osc_val[k]) if k < len(s.osc_val) else 0.0
        m.n_cores = s.n_cores
        m.core_power_idx = i(s.core_power_idx)
        m.n_true, m.e_lo, m.e_hi = s.n_true, s.e_lo, s.e_hi
        m.n_det = len(s.detectors)
        m.det_n_reco = i([dt.n_reco for dt in s.detectors])
        m.det_response = d(np.concatenate([dt.response.ravel() for dt in s.detectors]))
        ds = s.datasets
        m.n_ds = len(ds)
        m.ds_det = i([x.det for x in ds])
        m.ds_t = d(np.concatenate([x.t for x in ds]))
        m.ds_baseline = d(np.concatenate([x.baseline for x in ds]))
        m.ds_weight = d(np.concatenate([x.weight for x in ds]))
        m.ds_norm_idx = i([x.norm_idx for x in ds])
        m.ds_eff_idx = i([x.eff_idx for x in ds])
        m.ds_escale_idx = i(np.concatenate([x.escale_idx for x in ds]))
        m.ds_shape_idx = i(np.concatenate([x.shape_idx for x in ds]))
        bk = [(di, b) for di, x in enumerate(ds) for b in x.backgrounds]
        m.n_bkg = len(bk)
        m.bkg_ds = i([di for di, _ in bk] or [0])
        m.bkg_template = d(np.concatenate([b.template for _, b in bk]) if bk else [0.0])
        m.bkg_rate_idx = i([b.rate_idx for _, b in bk] or [0])
        m.bkg_shape_idx = i(np.concatenate([b.shape_idx for _, b in bk]) if bk else [0])
        h = C.c_void_p()
        _check(L.fit_model_create(C.byref(m), C.byref(h)), "fit_model_create")
        self._attach(h)

    def _attach(self, h):
        self.handle = h
        info = fit_model_info_t()
        _check(load().fit_model_info(h, C.byref(info)), "fit_model_info")
        self.n_params, self.n_data = info.n_params, info.n_data
        self.n_datasets, self.device_bytes = info.n_datasets, info.device_bytes

    @classmethod
    def from_json(cls, text, spec=None):
        """Model from a JSON configuration (str, bytes or a dict); `spec` is kept as metadata."""
        if isinstance(text, dict):
            import json
            text = json.dumps(text)
        if isinstance(text, str):
            text = text.encode()
        h = C.c_void_p()
        _check(load().fit_model_create_json(text, C.byref(h)), "fit_model_create_json")
        return cls(spec, _handle=h)

    def params(self):
        """(theta0, prior_sigma) host arrays kept by the library."""
        th, sg = np.zeros(self.n_params), np.zeros(self.n_params)
        _check(load().fit_model_params(self.handle, th.ctypes.data, sg.ctypes.data), "fit_model_params")
        return th, sg

    def param_names(self):
        """Parameter names kept by the library (None for a model built from a description)."""
        L = load()
        out = [L.fit_model_param_name(self.handle, i) for i in range(self.n_params)]
        return None if out[0] is None else [x.decode() for x in out]

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fit_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def fit_model_create(spec) -> Model:
    return Model(spec)


def fit_model_create_json(text, spec=None) -> Model:
    return Model.from_json(text, spec)


def fit_result_json(model: Model, best, result) -> str:
    """The library's JSON record of one fit: best = [n_params] float64 host array, result = one
    RESULT_DTYPE record (or a fit_result)."""
    best = np.ascontiguousarray(best, dtype=np.float64)
    if best.shape != (model.n_params,):
        raise ValueError("best must hold n_params values")
    r = np.ascontiguousarray(np.asarray(result).reshape(1), dtype=RESULT_DTYPE)
    L, n = load(), C.c_size_t()
    _check(L.fit_result_json(model.handle, best.ctypes.data, r.ctypes.data, None, 0, C.byref(n)),
           "fit_result_json")
    buf = C.create_string_buffer(n.value)
    _check(L.fit_result_json(model.handle, best.ctypes.data, r.ctypes.data, buf, n.value, C.byref(n)),
           "fit_result_json")
    return buf.value.decode()


def fit_model_destroy(model: Model):
    model.close()


def fit_model_expected(model: Model, B: int, theta, mu_out, status_out=None, stream=None):
    _check(load().fit_model_expected(model.handle, int(B), _ptr(theta), _ptr(mu_out),
                                     _ptr(status_out), _stream_ptr(stream)),
           "fit_model_expected")


def fit_model_eval(model: Model, B: int, theta, data, masks, nll_out, grad_out=None,
                   status_out=None, stream=None):
    if masks is not None and not hasattr(masks, "data_ptr"):
        masks = np.ascontiguousarray(masks, dtype=np.uint32)
    _check(load().fit_model_eval(model.handle, int(B), _ptr(theta), _ptr(data), _ptr(masks),
                                 _ptr(nll_out), _ptr(grad_out), _ptr(status_out),
                                 _stream_ptr(stream)),
           "fit_model_eval")


def fit_model_eval_noalloc(model: Model, B: int, theta, data, masks, nll_out, grad_out=None,
                           status_out=None, stream=None):
    """fit_model_eval without any device allocation (all buffers must be device memory)."""
    _check(load().fit_model_eval_noalloc(model.handle, int(B), _ptr(theta), _ptr(data),
                                         _ptr(masks), _ptr(nll_out), _ptr(grad_out),
                                         _ptr(status_out), _stream_ptr(stream)),
           "fit_model_eval_noalloc")


def fit_batch_default_opts() -> fit_batch_opts:
    o = fit_batch_opts()
    load().fit_batch_default_opts(C.byref(o))
    return o


def fit_batch(models, inst, data, start, best, results, opts=None, stream=None, fixed=None):
    """inst: numpy structured array of INSTANCE_DTYPE; results: RESULT_DTYPE array or a
    uint8 device tensor of n_inst * 32 bytes; fixed: optional uint8 flags indexed like start
    (held parameters, fit_batch_ex)."""
    L = load()
    hs = (C.c_void_p * len(models))(*[m.handle.value for m in models])
    inst = np.ascontiguousarray(inst, dtype=INSTANCE_DTYPE)
    o = opts if opts is not None else fit_batch_default_opts()
    if fixed is None:
        _check(L.fit_batch(hs, len(models), inst.ctypes.data, len(inst), _ptr(data), _ptr(start),
                           _ptr(best), _ptr(results), C.byref(o), _stream_ptr(stream)),
               "fit_batch")
    else:
        if not hasattr(fixed, "data_ptr"):
            fixed = np.ascontiguousarray(fixed, dtype=np.uint8)
        _check(L.fit_batch_ex(hs, len(models), inst.ctypes.data, len(inst), _ptr(data),
                              _ptr(start), _ptr(fixed), _ptr(best), _ptr(results), C.byref(o),
                              _stream_ptr(stream)),
               "fit_batch_ex")


def fit_profile_scan(model: Model, data, mask, scan_idx, points, start=None, opts=None,
                     stream=None):
    """Profile likelihood on a raster; returns dict(nll_min, theta_best, dchi2, theta, status)."""
    idx = np.ascontiguousarray(scan_idx, dtype=np.int32)
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, len(idx)))
    n = len(pts)
    P = model.n_params
    nll = C.c_double()
    tb = np.zeros(P)
    dchi2 = np.zeros(n)
    th = np.zeros((n, P))
    st = np.zeros(n, np.int32)
    if data is not None and not hasattr(data, "data_ptr"):
        data = np.ascontiguousarray(data, dtype=np.float32)
    if start is not None and not hasattr(start, "data_ptr"):
        start = np.ascontiguousarray(start, dtype=np.float64)
    o = opts if opts is not None else fit_batch_default_opts()
    _check(load().fit_profile_scan(model.handle, _ptr(data), C.c_uint32(int(mask)), len(idx),
                                   _ptr(idx), n, _ptr(pts), _ptr(start), C.byref(o),
                                   C.byref(nll), _ptr(tb), _ptr(dchi2), _ptr(th), _ptr(st),
                                   _stream_ptr(stream)),
           "fit_profile_scan")
    return dict(nll_min=nll.value, theta_best=tb, dchi2=dchi2, theta=th, status=st)


def fit_wilks_interval(x, dchi2, level=1.0):
    """(lo, hi, open_flags) where the 1-D profile dchi2(x) crosses `level`."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    d = np.ascontiguousarray(dchi2, dtype=np.float64)
    lo, hi = C.c_double(), C.c_double()
    rc = load().fit_wilks_interval(len(x), _ptr(x), _ptr(d), float(level), C.byref(lo),
                                   C.byref(hi))
    if rc < 0:
        _check(rc, "fit_wilks_interval")
    return lo.value, hi.value, rc


def fit_chi2_sf(chi2, dof):
    return float(load().fit_chi2_sf(float(chi2), int(dof)))


def fit_batch_autotune(models, inst, data, start=None, n_sample=0, opts=None, stream=None):
    """Times the fit kernel's launch configurations on a sample; returns the tuned options."""
    L = load()
    hs = (C.c_void_p * len(models))(*[m.handle.value for m in models])
    inst = np.ascontiguousarray(inst, dtype=INSTANCE_DTYPE)
    o = opts if opts is not None else fit_batch_default_opts()
    _check(L.fit_batch_autotune(hs, len(models), inst.ctypes.data, len(inst), _ptr(data),
                                _ptr(start), int(n_sample), C.byref(o), _stream_ptr(stream)),
           "fit_batch_autotune")
    return o


def fit_tc_gemm(tf32, M, N, K, A, lda, B, ldb, epi, C=None, ldc=0, Y=None, ldy=0, bias=None,
                aux=None, ldaux=0, stream=None):
    """Tensor-core GEMM D = A B^T with a fused epilogue (device buffers)."""
    _check(load().fit_tc_gemm(int(tf32), int(M), int(N), int(K), _ptr(A), int(lda), _ptr(B), int(ldb),
                              int(epi), _ptr(C), int(ldc), _ptr(Y), int(ldy), _ptr(bias), _ptr(aux),
                              int(ldaux), _stream_ptr(stream)), "fit_tc_gemm")


def fit_tc_gemm_status() -> int:
    return int(load().fit_tc_gemm_status())


def fit_kernel_launches() -> int:
    return int(load().fit_kernel_launches())


def fit_model_expected_tc(model: Model, B: int, theta, mu_out, status_out=None, precision=1,
                          stream=None):
    """Expected counts with the response fold on tensor cores (precision 0: TF32, 1: 3xTF32)."""
    _check(load().fit_model_expected_tc(model.handle, int(B), _ptr(theta), _ptr(mu_out),
                                        _ptr(status_out), int(precision), _stream_ptr(stream)),
           "fit_model_expected_tc")


def fit_poisson_sample(n, mu, seed, offset, out, stream=None):
    """out[i] ~ Poisson(mu[i]) (float32), Philox4x32-10 counters (i + offset, draw)."""
    _check(load().fit_poisson_sample(int(n), _ptr(mu), C.c_uint64(int(seed) & (2**64 - 1)),
                                     C.c_uint64(int(offset)), _ptr(out), _stream_ptr(stream)),
           "fit_poisson_sample")


class McEventSet:
    """Simulated signal events of one detector resident on the current CUDA device (wraps
    fit_mc*). events: an object with energy, core, weight, bin (sorted), n_bins, core_L and
    osc_mode, e.g. synth.McEvents."""

    def __init__(self, events):
        e = np.ascontiguousarray(events.energy, dtype=np.float32)
        c = np.ascontiguousarray(events.core, dtype=np.uint8)
        w = np.ascontiguousarray(events.weight, dtype=np.float32)
        b = np.ascontiguousarray(events.bin, dtype=np.int32)
        L = np.ascontiguousarray(events.core_L, dtype=np.float64)
        if not (len(e) == len(c) == len(w) == len(b)):
            raise ValueError("event arrays differ in length")
        h = C.c_void_p()
        _check(load().fit_mc_create(int(events.osc_mode), len(L), _ptr(L), len(e), _ptr(e), _ptr(c),
                                    _ptr(w), _ptr(b), int(events.n_bins), C.byref(h)),
               "fit_mc_create")
        self.handle = h
        self.n_events, self.n_bins = len(e), int(events.n_bins)

    def spectrum(self, B, params, out, stream=None):
        """out[b, j] = sum of w_e P(L_e, E_e; params[b]) over the events of bin j (float64 [B x
        n_bins]; params float64 [B x 4]; host or device buffers)."""
        _check(load().fit_mc_spectrum(self.handle, int(B), _ptr(params), _ptr(out),
                                      _stream_ptr(stream)), "fit_mc_spectrum")

    def status(self):
        """Raises FitError if a staging wait of an earlier spectrum call ran out of time."""
        _check(load().fit_mc_status(self.handle), "fit_mc_status")

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fit_mc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


class Mlp:
    """Warm-start network resident on the current CUDA device (wraps fit_mlp*)."""

    def __init__(self, n_in, n_hidden, n_hidden_layers, n_out, seed=0):
        h = C.c_void_p()
        _check(load().fit_mlp_create(int(n_in), int(n_hidden), int(n_hidden_layers), int(n_out),
                                     C.c_uint64(int(seed)), C.byref(h)), "fit_mlp_create")
        self.handle = h
        self.n_in, self.n_hidden, self.n_out = int(n_in), int(n_hidden), int(n_out)
        self.n_layers = int(n_hidden_layers) + 1

    def layer_shape(self, layer):
        fan_in = self.n_in if layer == 0 else self.n_hidden
        fan_out = self.n_out if layer == self.n_layers - 1 else self.n_hidden
        return fan_out, fan_in

    def forward(self, B, x, y, stream=None):
        _check(load().fit_mlp_forward(self.handle, int(B), _ptr(x), _ptr(y), _stream_ptr(stream)),
               "fit_mlp_forward")

    def train_step(self, B, x, target, lr, weight_decay=0.0, loss_out=None, stream=None):
        _check(load().fit_mlp_train_step(self.handle, int(B), _ptr(x), _ptr(target), float(lr),
                                         float(weight_decay), _ptr(loss_out), _stream_ptr(stream)),
               "fit_mlp_train_step")

    def get_layer(self, layer):
        o, i = self.layer_shape(layer)
        w, b = np.zeros((o, i), np.float32), np.zeros(o, np.float32)
        gw, gb = np.zeros((o, i), np.float32), np.zeros(o, np.float32)
        _check(load().fit_mlp_get_layer(self.handle, int(layer), _ptr(w), _ptr(b), _ptr(gw),
                                        _ptr(gb)), "fit_mlp_get_layer")
        return w, b, gw, gb

    def set_layer(self, layer, w, b):
        o, i = self.layer_shape(layer)
        w = np.ascontiguousarray(w, dtype=np.float32).reshape(o, i)
        b = np.ascontiguousarray(b, dtype=np.float32).reshape(o)
        _check(load().fit_mlp_set_layer(self.handle, int(layer), _ptr(w), _ptr(b)),
               "fit_mlp_set_layer")

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fit_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def fit_warmstart_features(model: Model, B, data, masks, n_in, slot0, onehot_slot, x, stream=None):
    _check(load().fit_warmstart_features(model.handle, int(B), _ptr(data), _ptr(masks), int(n_in),
                                         int(slot0), int(onehot_slot), _ptr(x),
                                         _stream_ptr(stream)),
           "fit_warmstart_features")


def fit_warmstart_predict(mlp: Mlp, model: Model, B, data, masks, slot0, onehot_slot, target_idx,
                          target_scale, theta_out, stream=None):
    """Start points: the linearised best fit of every parameter plus the network's corrections
    on its targets."""
    idx = np.ascontiguousarray(target_idx, dtype=np.int32)
    scl = np.ascontiguousarray(target_scale, dtype=np.float64)
    _check(load().fit_warmstart_predict(mlp.handle, model.handle, int(B), _ptr(data), _ptr(masks),
                                        int(slot0), int(onehot_slot), len(idx), _ptr(idx),
                                        _ptr(scl), _ptr(theta_out), _stream_ptr(stream)),
           "fit_warmstart_predict")


def fit_linear_start(model: Model, B, data, masks, theta_out, stream=None):
    """Start points theta_out [B x P] (device) from the linearised best fit: one Gauss-Newton
    step of -2lnL from theta0 with the expected Hessian (device data [B x n_data]; masks host
    or device [B] or None)."""
    _check(load().fit_linear_start(model.handle, int(B), _ptr(data), _ptr(masks), _ptr(theta_out),
                                   _stream_ptr(stream)), "fit_linear_start")


def make_geom(slot0, onehot_slot, target_idx, target_scale, uniform_idx=(), uniform_half=(),
              masks=()) -> fit_warmstart_geom:
    g = fit_warmstart_geom()
    g.slot0, g.onehot_slot = int(slot0), int(onehot_slot)
    if not (0 < len(target_idx) <= WS_MAX_TARGETS and len(target_scale) == len(target_idx)
            and len(uniform_idx) == len(uniform_half) and len(uniform_idx) <= WS_MAX_TARGETS
            and len(masks) <= WS_MAX_MASKS):
        raise ValueError("warm-start geometry: table sizes")
    g.n_targets = len(target_idx)
    for t, (i, sc) in enumerate(zip(target_idx, target_scale)):
        g.target_idx[t], g.target_scale[t] = int(i), float(sc)
    g.n_uniform = len(uniform_idx)
    for t, (i, h) in enumerate(zip(uniform_idx, uniform_half)):
        g.uniform_idx[t], g.uniform_half[t] = int(i), float(h)
    g.n_masks = len(masks)
    for t, mk in enumerate(masks):
        g.masks[t] = int(mk)
    return g


def fit_warmstart_draw(model: Model, geom: fit_warmstart_geom, B, seed, offset, theta_out,
                       masks_out=None, stream=None):
    _check(load().fit_warmstart_draw(model.handle, C.byref(geom), int(B), C.c_uint64(int(seed)),
                                     C.c_uint64(int(offset)), _ptr(theta_out), _ptr(masks_out),
                                     _stream_ptr(stream)),
           "fit_warmstart_draw")


def fit_warmstart_train(mlp: Mlp, models, geoms, n_steps, batch, lr, weight_decay, seed,
                        losses_out=None, stream=None):
    hs = (C.c_void_p * len(models))(*[m.handle.value for m in models])
    gs = (fit_warmstart_geom * len(geoms))(*geoms)
    _check(load().fit_warmstart_train(mlp.handle, hs, gs, len(geoms), int(n_steps), int(batch),
                                      float(lr), float(weight_decay), C.c_uint64(int(seed)),
                                      _ptr(losses_out), _stream_ptr(stream)),
           "fit_warmstart_train")


# ---- convenience wrappers used by tests and the benchmark ---------------------------------
def eval_numpy(model: Model, theta, data=None, masks=None, grad=True):
    """-2lnL (and gradient) for a [B, P] float64 array, host buffers in and out."""
    theta = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
    B = theta.shape[0]
    if data is not None:
        data = np.ascontiguousarray(np.atleast_2d(data), dtype=np.float32)
    nll = np.zeros(B)
    g = np.zeros((B, model.n_params), np.float32) if grad else None
    st = np.zeros(B, np.int32)
    fit_model_eval(model, B, theta, data, masks, nll, g, st)
    return nll, g, st


def expected_numpy(model: Model, theta):
    theta = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
    mu = np.zeros((theta.shape[0], model.n_data), np.float32)
    st = np.zeros(theta.shape[0], np.int32)
    fit_model_expected(model, theta.shape[0], theta, mu, st)
    return mu, st


def fit_numpy(models, inst, data, start=None, opts=None, fixed=None):
    """Runs fit_batch on host arrays; returns (best [flat float64], results RESULT_DTYPE)."""
    inst = np.ascontiguousarray(inst, dtype=INSTANCE_DTYPE)
    npar = max(int(r["param_off"]) + models[int(r["model"])].n_params for r in inst)
    best = np.zeros(npar)
    res = np.zeros(len(inst), RESULT_DTYPE)
    data = np.ascontiguousarray(data, dtype=np.float32)
    if start is not None:
        start = np.ascontiguousarray(start, dtype=np.float64)
    fit_batch(models, inst, data, start, best, res, opts, fixed=fixed)
    return best, res


# ---- torch autograd wrapper ------------------------------------------------------------------
def _autograd_function():
    import torch

    class FitNLL(torch.autograd.Function):
        """-2lnL of a batch of parameter vectors as a differentiable torch op.

        forward(theta [B, P] float64 CUDA tensor, data [B, n_data] float32 CUDA tensor or None
        (the model's Asimov data), model, masks [B] uint32 tensor or None) -> nll [B] float64.
        The gradient comes from the library's adjoint (fit_model_eval); backward returns
        grad_output[:, None] * d(-2lnL)/dtheta.
        """

        @staticmethod
        def forward(ctx, theta, data, model, masks=None):
            if not (theta.is_cuda and theta.dtype == torch.float64 and theta.dim() == 2):
                raise ValueError("theta must be a [B, P] float64 CUDA tensor")
            th = theta.detach().contiguous()
            B = th.shape[0]
            nll = torch.empty(B, dtype=torch.float64, device=th.device)
            grad = torch.empty((B, model.n_params), dtype=torch.float32, device=th.device)
            dd = data.detach().contiguous() if data is not None else None
            fit_model_eval(model, B, th, dd, masks, nll, grad)
            ctx.save_for_backward(grad)
            return nll

        @staticmethod
        def backward(ctx, grad_out):
            (grad,) = ctx.saved_tensors
            return grad_out[:, None] * grad.to(grad_out.dtype), None, None, None

    return FitNLL


def fit_nll(theta, data, model, masks=None):
    """Differentiable -2lnL (see FitNLL)."""
    return _autograd_function().apply(theta, data, model, masks)
