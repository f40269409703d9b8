"""FP64 CPU oracle of the forward-folding likelihood fit - TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import this package. The CUDA library never calls it, and the two share no code: this
wrapper only marshals the seeded inputs of ``paper_2502_15253_gb300.synth`` into the C
structures of ``oracle.c`` (its own definitions) and calls the plain FP64 implementation.

Parity status per function (what pins it is in tests/test_oracle_pins.py):
  survival (Eq. 1 / 3-flavour vacuum) - pinned (zero mixing, 2-flavour limit, brute-force
      PMNS amplitude, corrected Eq. 10, Eq. 1 vs exact bound)
  remap (energy correction)           - pinned (identity, shift by whole bins, conservation,
      brute-force fine-grid integration)
  deviance / nll / gradient           - pinned (closed forms, Asimov zero, central FD,
      hand-summed toy model)
  fit (BFGS)                          - pinned (Asimov recovery, pure-scale closed form,
      prior-only closed form, brute-force grid scan on a 2-parameter model)
  sigma (FD Hessian)                  - pinned (prior-only model: 2 H^-1 = V exactly)
  event_spectrum (event reweighting)  - pinned (zero mixing = weighted bin counts; per-event
      sum of the pinned survival function on a small sample)
  philox4x32_10 (rng.c)               - pinned (published known-answer vectors)
  poisson_sample (rng.c)              - pinned (chi-square against the exact Poisson PMF,
      mean and variance, counter/offset invariance)
  linear_prior_block (Eq. 6, b = A theta) - pinned (the quadratic forms agree at random points
      up to one constant; A = identity returns (b0, V, 0); a direct search for the minimum)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "rng.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

STATUS = {0: "converged", 1: "maxiter", 2: "linesearch_fail", 3: "nonfinite",
          4: "fixed parameter inside a prior block"}


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *_SRCS, "-o",
            tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


class _OrcModel(C.Structure):
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
        ("n_map", C.c_int),
        ("map_k", C.POINTER(C.c_int)), ("map_m", C.POINTER(C.c_int)),
        ("map_idx", C.POINTER(C.c_int)),
        ("map_A", C.POINTER(C.c_double)), ("map_b0", C.POINTER(C.c_double)),
        ("map_V", C.POINTER(C.c_double)),
    ]


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)


def _declare(L):
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.POINTER(_OrcModel)]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_n_data.restype = C.c_int
    L.orc_n_data.argtypes = [C.c_void_p]
    L.orc_survival.restype = C.c_double
    L.orc_survival.argtypes = [C.c_int, _DP, C.c_double, C.c_double, _DP]
    L.orc_remap.restype = C.c_int
    L.orc_remap.argtypes = [C.POINTER(_OrcModel), _DP, _DP, _DP]
    L.orc_expected.restype = C.c_int
    L.orc_expected.argtypes = [C.c_void_p, _DP, _DP]
    L.orc_deviance.restype = C.c_double
    L.orc_deviance.argtypes = [C.c_double, C.c_double]
    L.orc_nll.restype = C.c_double
    L.orc_nll.argtypes = [C.c_void_p, _DP, _DP, C.c_uint32, _DP]
    L.orc_theta_of_z.argtypes = [C.c_void_p, _DP, _DP]
    L.orc_z_of_theta.argtypes = [C.c_void_p, _DP, _DP]
    L.orc_fit.restype = C.c_int
    L.orc_fit.argtypes = [C.c_void_p, _DP, C.c_uint32, _DP, C.c_double, C.c_int, _DP, _DP, _IP,
                          _IP, _DP]
    L.orc_fit_ex.restype = C.c_int
    L.orc_fit_ex.argtypes = [C.c_void_p, _DP, C.c_uint32, _DP, C.POINTER(C.c_ubyte), C.c_double,
                             C.c_int, _DP, _DP, _IP, _IP, _DP]
    L.orc_fit_many.argtypes = [C.POINTER(C.c_void_p), C.c_int, _IP, C.POINTER(_DP),
                               C.POINTER(C.c_uint32), C.POINTER(_DP), C.c_double, C.c_int,
                               C.POINTER(_DP), _DP, _IP, _IP, _IP, C.c_int]
    L.orc_openmp_enabled.restype = C.c_int
    L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    L.orc_philox4x32_10.restype = None
    L.orc_poisson_sample.argtypes = [C.c_int64, C.POINTER(C.c_float), C.c_uint64, C.c_uint64,
                                     C.POINTER(C.c_float)]
    L.orc_poisson_sample.restype = None
    L.orc_ptrs_step_many.argtypes = [C.c_float, C.c_int64, C.POINTER(C.c_float),
                                     C.POINTER(C.c_float), C.POINTER(C.c_float)]
    L.orc_ptrs_step_many.restype = None
    L.orc_event_spectrum.argtypes = [C.c_int, _DP, _DP, C.c_longlong, C.POINTER(C.c_float),
                                     C.POINTER(C.c_ubyte), C.POINTER(C.c_float), _IP, C.c_int, _DP]
    L.orc_event_spectrum.restype = None


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_DP)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_IP)


def survival(mode: int, p, L: float, E: float, with_grad: bool = False):
    """Survival probability P(L, E) (Eq. 1 for mode 0, exact 3-flavour vacuum for mode 1, exact
    3+1 vacuum for mode 2 with p = (sin^2 th12, sin^2 th13, dm2_21, dm2_31, sin^2 2th14, dm2_41))."""
    n = 6 if int(mode) == 2 else 4
    p = np.ascontiguousarray(p, dtype=np.float64)
    if p.size != n:
        raise ValueError(f"mode {mode} takes {n} parameters")
    pa, pp = _d(p)
    dp = np.zeros(n)
    val = lib().orc_survival(int(mode), pp, float(L), float(E), _d(dp)[1] if with_grad else None)
    if with_grad:
        # _d returned a view of dp (already float64 contiguous), so dp was written in place
        return val, dp
    return val


def deviance(n: float, mu: float) -> float:
    return lib().orc_deviance(float(n), float(mu))


class OracleModel:
    """A ModelSpec marshalled into the oracle's C structure."""

    def __init__(self, spec):
        self.spec = spec
        keep = []

        def d(a):
            arr, ptr = _d(a)
            keep.append(arr)
            return ptr

        def i(a):
            arr, ptr = _i(a)
            keep.append(arr)
            return ptr

        s = spec
        m = _OrcModel()
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
        m.n_ds = len(s.datasets)
        ds = s.datasets
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
        # Eq. 6 priors on b = A theta (evaluated as written, not converted)
        mp = list(getattr(s, "map_priors", []) or [])
        m.n_map = len(mp)
        m.map_k = i([len(ix) for ix, _, _, _ in mp] or [0])
        m.map_m = i([len(b0) for _, _, b0, _ in mp] or [0])
        m.map_idx = i(np.concatenate([np.asarray(ix) for ix, _, _, _ in mp]) if mp else [0])
        m.map_A = d(np.concatenate([np.asarray(A, np.float64).ravel() for _, A, _, _ in mp]) if mp else [0.0])
        m.map_b0 = d(np.concatenate([np.asarray(b0, np.float64) for _, _, b0, _ in mp]) if mp else [0.0])
        m.map_V = d(np.concatenate([np.asarray(V, np.float64).ravel() for _, _, _, V in mp]) if mp else [0.0])
        for ix, A, b0, V in mp:
            if np.shape(A) != (len(b0), len(ix)) or np.shape(V) != (len(b0), len(b0)):
                raise ValueError("oracle: a map prior needs A [m x k], b0 [m] and V [m x m]")
        self._keep = keep
        self._m = m
        self.h = lib().orc_create(C.byref(m))
        if not self.h:
            raise ValueError("oracle: a prior covariance (block or map) is not symmetric positive "
                             "definite")
        self.n_params = s.n_params
        self.n_data = lib().orc_n_data(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self.h = None

    # -- forward model ------------------------------------------------------------------
    def expected(self, theta) -> np.ndarray:
        th, tp = _d(theta)
        mu = np.zeros(self.n_data)
        st = lib().orc_expected(self.h, tp, mu.ctypes.data_as(_DP))
        if st:
            raise ValueError("oracle: energy map not increasing on the grid")
        return mu

    def nll(self, theta, data, mask=None, grad=False):
        th, tp = _d(theta)
        da, dp = _d(data)
        mask = self.spec.all_mask() if mask is None else mask
        if grad:
            g = np.zeros(self.n_params)
            v = lib().orc_nll(self.h, tp, dp, C.c_uint32(mask), g.ctypes.data_as(_DP))
            return v, g
        return lib().orc_nll(self.h, tp, dp, C.c_uint32(mask), None)

    def remap(self, a, u) -> np.ndarray:
        aa, ap = _d(a)
        ua, up = _d(u)
        v = np.zeros(self.spec.n_true)
        st = lib().orc_remap(C.byref(self._m), ap, up, v.ctypes.data_as(_DP))
        if st:
            raise ValueError("oracle: energy map not increasing on the grid")
        return v

    # -- transformation layer -----------------------------------------------------------
    def theta_of_z(self, z):
        za, zp = _d(z)
        th = np.zeros(self.n_params)
        lib().orc_theta_of_z(self.h, zp, th.ctypes.data_as(_DP))
        return th

    def z_of_theta(self, theta):
        ta, tp = _d(theta)
        z = np.zeros(self.n_params)
        lib().orc_z_of_theta(self.h, tp, z.ctypes.data_as(_DP))
        return z

    # -- minimiser ----------------------------------------------------------------------
    def fit(self, data, mask=None, start=None, edm_tol=1e-10, max_iter=5000, fixed=None):
        """Dense BFGS fit. Returns dict(theta, nll, iters, nevals, edm, status).

        fixed: optional boolean array over the parameters held at their start values (the
        constrained fit of a profile likelihood); parameters inside a prior block cannot be
        fixed (status 4)."""
        mask = self.spec.all_mask() if mask is None else mask
        start = self.spec.theta0 if start is None else start
        da, dp = _d(data)
        sa, sp = _d(start)
        th = np.zeros(self.n_params)
        nll, edm = C.c_double(), C.c_double()
        it, ne = C.c_int(), C.c_int()
        fx = None
        if fixed is not None:
            fa = np.ascontiguousarray(np.asarray(fixed, dtype=bool), dtype=np.uint8)
            fx = fa.ctypes.data_as(C.POINTER(C.c_ubyte))
        st = lib().orc_fit_ex(self.h, dp, C.c_uint32(mask), sp, fx, edm_tol, max_iter,
                              th.ctypes.data_as(_DP), C.byref(nll), C.byref(it), C.byref(ne),
                              C.byref(edm))
        return dict(theta=th, nll=nll.value, iters=it.value, nevals=ne.value, edm=edm.value,
                    status=st)

    def hessian(self, theta, data, mask=None, rel_step=1e-3):
        """Hessian of -2lnL in theta, by central differences of the analytic gradient.

        Steps are rel_step times each parameter's minimiser scale; the result is symmetrised.
        """
        n = self.n_params
        h = np.where(self.spec.prior_sigma > 0, self.spec.prior_sigma, self.spec.scale) * rel_step
        H = np.zeros((n, n))
        for i in range(n):
            tp = np.array(theta, np.float64)
            tm = tp.copy()
            tp[i] += h[i]
            tm[i] -= h[i]
            gp = self.nll(tp, data, mask, grad=True)[1]
            gm = self.nll(tm, data, mask, grad=True)[1]
            H[:, i] = (gp - gm) / (2.0 * h[i])
        return 0.5 * (H + H.T)

    def sigma(self, theta, data, mask=None, rel_step=1e-3):
        """Parameter errors sqrt(2 (H^-1)_ii) at theta (H = Hessian of -2lnL).

        Parameters with no curvature (no data and no prior) get +inf.
        """
        H = self.hessian(theta, data, mask, rel_step)
        live = np.abs(np.diag(H)) > 1e-300
        sig = np.full(self.n_params, np.inf)
        if live.any():
            # At a kink of the energy correction the difference Hessian can have a slightly
            # negative eigenvalue; inverting its projection onto the positive semidefinite
            # cone (eigenvalues floored at 1e-9 of the largest) keeps every sigma > 0.
            Hl = H[np.ix_(live, live)]
            w, V = np.linalg.eigh(Hl)
            w = np.maximum(w, 1e-9 * max(w.max(), 1e-300))
            sig[live] = np.sqrt(2.0 * np.einsum("ij,j,ij->i", V, 1.0 / w, V))
        return sig


def fit_many(models, model_of, data, masks, starts, edm_tol=1e-10, max_iter=5000, n_threads=None):
    """Fits many instances on host threads (OpenMP). models: list of OracleModel."""
    n = len(model_of)
    n_threads = n_threads or os.cpu_count() or 1
    hs = (C.c_void_p * len(models))(*[m.h for m in models])
    mo, mop = _i(model_of)
    keep = []
    dptr = (_DP * n)()
    sptr = (_DP * n)()
    optr = (_DP * n)()
    outs = []
    for i in range(n):
        a, p = _d(data[i])
        b, q = _d(starts[i])
        o = np.zeros(models[model_of[i]].n_params)
        keep += [a, b]
        outs.append(o)
        dptr[i], sptr[i], optr[i] = p, q, o.ctypes.data_as(_DP)
    mk = np.ascontiguousarray(masks, dtype=np.uint32)
    nll = np.zeros(n)
    iters = np.zeros(n, np.int32)
    nev = np.zeros(n, np.int32)
    st = np.zeros(n, np.int32)
    lib().orc_fit_many(hs, n, mop, dptr, mk.ctypes.data_as(C.POINTER(C.c_uint32)), sptr,
                       edm_tol, max_iter, optr, nll.ctypes.data_as(_DP),
                       iters.ctypes.data_as(_IP), nev.ctypes.data_as(_IP),
                       st.ctypes.data_as(_IP), int(n_threads))
    return dict(theta=outs, nll=nll, iters=iters, nevals=nev, status=st)


def openmp_enabled() -> bool:
    return bool(lib().orc_openmp_enabled())


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: four 32-bit output words for a 4-word counter and 2-word key."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    lib().orc_philox4x32_10(c, k)
    return [int(x) for x in c]


def poisson_sample(mu, seed: int, offset: int = 0):
    """Poisson draws (float32) for the float32 means mu; element i uses counter i + offset."""
    mu = np.ascontiguousarray(mu, dtype=np.float32).ravel()
    out = np.zeros_like(mu)
    lib().orc_poisson_sample(len(mu), mu.ctypes.data_as(C.POINTER(C.c_float)),
                             C.c_uint64(int(seed) & (2**64 - 1)), C.c_uint64(int(offset)),
                             out.ctypes.data_as(C.POINTER(C.c_float)))
    return out


def ptrs_step(mu: float, U, V):
    """One PTRS trial per (U, V) pair for mean mu >= 10: accepted count, or -1 if rejected."""
    U = np.ascontiguousarray(U, dtype=np.float32).ravel()
    V = np.ascontiguousarray(V, dtype=np.float32).ravel()
    k = np.zeros_like(U)
    F = C.POINTER(C.c_float)
    lib().orc_ptrs_step_many(float(mu), len(U), U.ctypes.data_as(F), V.ctypes.data_as(F),
                             k.ctypes.data_as(F))
    return k


def event_spectrum(events, params):
    """Oscillated spectrum of Monte Carlo events (synth.McEvents) at the survival parameters
    params[4], summed per reco bin in FP64."""
    e = np.ascontiguousarray(events.energy, dtype=np.float32)
    c = np.ascontiguousarray(events.core, dtype=np.uint8)
    w = np.ascontiguousarray(events.weight, dtype=np.float32)
    b = np.ascontiguousarray(events.bin, dtype=np.int32)
    pa, pp = _d(params)
    la, lp = _d(events.core_L)
    out = np.zeros(events.n_bins)
    lib().orc_event_spectrum(int(events.osc_mode), pp, lp, len(e),
                             e.ctypes.data_as(C.POINTER(C.c_float)),
                             c.ctypes.data_as(C.POINTER(C.c_ubyte)),
                             w.ctypes.data_as(C.POINTER(C.c_float)), b.ctypes.data_as(_IP),
                             int(events.n_bins), out.ctypes.data_as(_DP))
    return out


def linear_prior_block(A, b0, V):
    """Eq. 6 with a linear generalised parametrisation b(theta) = A theta: the Gaussian prior
    (A theta - b0)^T V^-1 (A theta - b0) written as a covariance block on theta,
    (theta - t)^T Cb^-1 (theta - t) + const. Expanding the quadratic form:
    Cb = (A^T V^-1 A)^-1, t = Cb A^T V^-1 b0, const = b0^T V^-1 b0 - t^T Cb^-1 t.
    Returns (t, Cb, const)."""
    A = np.asarray(A, dtype=np.float64)
    b0 = np.asarray(b0, dtype=np.float64)
    Vinv = np.linalg.inv(np.asarray(V, dtype=np.float64))
    F = A.T @ Vinv @ A
    Cb = np.linalg.inv(F)
    t = Cb @ (A.T @ Vinv @ b0)
    const = float(b0 @ Vinv @ b0 - t @ F @ t)
    return t, Cb, const
