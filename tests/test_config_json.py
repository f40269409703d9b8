"""Model creation from a JSON configuration (fit_model_create_json): the reader and the
mapping onto the model description are host code, so every rejection below happens before a
device call and runs on the CPU. ([S]: the framework reads a configuration file naming the
parameters, their priors and the datasets.)"""
import copy
import ctypes
import json

import numpy as np
import pytest

from paper_2502_15253_gb300 import fitcore, synth

INVALID_CONFIG = -2


def _create(text):
    """(rc, message, handle) of fit_model_create_json on a str / bytes configuration."""
    L = fitcore.load()
    h = ctypes.c_void_p()
    raw = text.encode() if isinstance(text, str) else text
    rc = L.fit_model_create_json(raw, ctypes.byref(h))
    msg = L.fit_last_error().decode() if rc else ""
    if rc == 0:   # only where a device is present
        L.fit_model_destroy(h)
    return rc, msg


def _reject(cfg):
    rc, msg = _create(json.dumps(cfg) if isinstance(cfg, dict) else cfg)
    assert rc == INVALID_CONFIG, (rc, msg)
    return msg


@pytest.fixture(scope="module")
def cfg():
    return synth.make_model("c0").to_config()


@pytest.mark.parametrize("text,where", [
    ("", "offset 0"), ("{", "offset 1"), ('{"a": }', "offset 6"), ('{"a" 1}', "expected ':'"),
    ('{"a": [1, 2}', "expected ',' or ']'"), ('{"a": "x}', "unterminated string"),
    ('{"a": 1} 2', "trailing characters"), ('{"a": tru}', "offset"), ('{"a": "\\q"}', "bad escape"),
    ("[" * 100 + "]" * 100, "nesting too deep"), ("[1, 2]", "must be an object"),
    ('{"a": "\\ud800"}', "unpaired surrogate"), ('{"a": "\\udc00x"}', "unpaired surrogate"),
    ('{"a": "\\u12G4"}', "bad \\u escape"),
])
def test_malformed_json_is_rejected_with_its_offset(text, where):
    assert where in _reject(text)


def test_null_arguments():
    L = fitcore.load()
    h = ctypes.c_void_p()
    assert L.fit_model_create_json(None, ctypes.byref(h)) == -1
    assert L.fit_model_create_json(b"{}", None) == -1
    assert L.fit_model_param_name(None, 0) is None


def _edit(cfg, fn):
    c = copy.deepcopy(cfg)
    fn(c)
    return c


@pytest.mark.parametrize("edit,where", [
    (lambda c: c.pop("parameters"), 'missing "parameters"'),
    (lambda c: c.pop("datasets"), 'missing "datasets"'),
    (lambda c: c["parameters"][3].pop("value"), "parameters[3]: missing \"value\""),
    (lambda c: c["parameters"][1].update(name=c["parameters"][0]["name"]), "duplicate name"),
    (lambda c: c["parameters"][2].update(sigma="wide"), "parameters[2].sigma: expected a number"),
    (lambda c: c["datasets"][0].update(norm="no_such"), 'unknown parameter "no_such"'),
    (lambda c: c["datasets"][0].update(efficiency=10**6), "datasets[0].efficiency: parameter index out of range"),
    (lambda c: c["datasets"][0].update(efficiency=1.5), "expected an integer"),
    (lambda c: c["datasets"][0].update(detector="nd"), 'unknown detector "nd"'),
    (lambda c: c["datasets"][0].update(detector=3), "datasets[0].detector: out of range"),
    (lambda c: c["datasets"][0]["t"].pop(), "datasets[0].t: expected true_grid.bins entries"),
    (lambda c: c["datasets"][0]["shape"].pop(), "datasets[0].shape"),
    (lambda c: c["datasets"][0]["escale"].pop(), "three entries"),
    (lambda c: c["datasets"][0]["baseline"].append(400.0), "one entry per core"),
    (lambda c: c["datasets"][0]["backgrounds"][0]["template"].pop(), "backgrounds[0].template"),
    (lambda c: c["datasets"][0]["backgrounds"][0].update(rate="x"), "backgrounds[0].rate"),
    (lambda c: c["detectors"][0]["response"][0].pop(), "detectors[0].response"),
    (lambda c: c["oscillation"].update(formula="eq2"), "oscillation.formula"),
    (lambda c: c["oscillation"]["params"].pop(), "expected 4 entries"),
    (lambda c: c["oscillation"]["params"].__setitem__(0, "nope"), 'unknown parameter "nope"'),
    (lambda c: c["oscillation"]["params"].__setitem__(0, [1]), "oscillation.params[0]: expected a number"),
    (lambda c: c.update(energy_correction="cubic"), "energy_correction"),
    (lambda c: c["true_grid"].update(bins=0.5), "true_grid.bins: expected an integer"),
    (lambda c: c["covariances"][0]["cov"].pop(), "covariances[0].cov"),
    (lambda c: c["covariances"][0]["params"].__setitem__(0, None), "null is not a parameter"),
    # caught by the description's own validation, still before any device call
    (lambda c: c["true_grid"].update(e_lo=20.0), "energy grid"),
    (lambda c: c["parameters"][0].update(sigma=-1.0), "prior_sigma"),
])
def test_configuration_errors_name_the_field(cfg, edit, where):
    assert where in _reject(_edit(cfg, edit))


def test_config_round_trips_the_description():
    """The configuration written by ModelSpec.to_config carries every array of the
    description exactly (JSON numbers are printed to round-trip FP64)."""
    for name in ["c0", "c1", "c1s"]:
        s = synth.make_model(name, remap=1 if name == "c1" else 0)
        c = json.loads(s.to_json())
        ix = {p["name"]: i for i, p in enumerate(c["parameters"])}
        assert [p["name"] for p in c["parameters"]] == list(s.param_names)
        assert np.array_equal([p["value"] for p in c["parameters"]], s.theta0)
        assert np.array_equal([p["sigma"] for p in c["parameters"]], s.prior_sigma)
        assert c["energy_correction"] == ("spline" if name == "c1" else "overlap")
        for k, e in enumerate(c["oscillation"]["params"]):
            if isinstance(e, str):
                assert ix[e] == s.osc_idx[k]
            else:
                assert s.osc_idx[k] == -1 and e == s.osc_val[k]
        for d, x in zip(c["datasets"], s.datasets):
            assert np.array_equal(d["t"], x.t)
            assert [ix[n] if n else -1 for n in d["shape"]] == list(x.shape_idx)
            for b, y in zip(d["backgrounds"], x.backgrounds):
                assert np.array_equal(b["template"], y.template)
        for dt, y in zip(c["detectors"], s.detectors):
            assert np.array_equal(np.asarray(dt["response"]), y.response)


def test_valid_configuration_reaches_the_device_step(cfg):
    """A valid configuration passes every host check: without a device the first error is the
    allocation's (OOM or CUDA); with one the model is created."""
    rc, msg = _create(json.dumps(cfg))
    assert rc in (0, -4, -6), (rc, msg)
    if rc:
        assert msg.startswith("fit_model_create:") and "cuda" in msg.lower()


def test_result_json_and_params_reject_null_arguments():
    L = fitcore.load()
    n = ctypes.c_size_t()
    assert L.fit_result_json(None, None, None, None, 0, ctypes.byref(n)) == -1
    assert "null argument" in L.fit_last_error().decode()
    assert L.fit_model_params(None, None, None) == -1


def test_covariance_blocks_must_be_symmetric_positive_definite(cfg):
    """Eq. 6: a covariance prior needs V_B symmetric positive definite (its Cholesky factor is
    the transformation layer); either failure is NON_SPD_COV, found on the host."""
    NON_SPD = -3
    c = copy.deepcopy(cfg)
    cov = np.asarray(c["covariances"][0]["cov"])
    m = len(cov)
    assert m >= 2
    asym = cov.copy()
    asym[0, 1] += 0.1 * np.sqrt(cov[0, 0] * cov[1, 1])
    c["covariances"][0]["cov"] = asym.tolist()
    rc, msg = _create(json.dumps(c))
    assert rc == NON_SPD and "symmetric" in msg
    # symmetric but indefinite: a negative eigenvalue
    w, v = np.linalg.eigh(cov)
    w[0] = -abs(w[-1])
    c["covariances"][0]["cov"] = ((v * w) @ v.T).tolist()
    rc, msg = _create(json.dumps(c))
    assert rc == NON_SPD and "positive definite" in msg


def test_non_finite_inputs_are_rejected(cfg):
    """JSON has no NaN or infinity: such a number (as Python writes it) is malformed JSON; in a
    description a non-finite response entry is a configuration error."""
    c = _edit(cfg, lambda c: c["detectors"][0]["response"][3].__setitem__(5, float("nan")))
    assert "expected a value" in _reject(json.dumps(c))
    c = _edit(cfg, lambda c: c["datasets"][0]["t"].__setitem__(2, float("inf")))
    assert "expected a value" in _reject(json.dumps(c))
    s2 = copy.deepcopy(synth.make_model("c0"))
    s2.detectors[0].response[3, 5] = np.nan
    with pytest.raises(fitcore.FitError, match="finite"):
        fitcore.Model(s2)


@pytest.mark.parametrize("mutate,where", [
    (lambda s: s.theta0.__setitem__(0, np.inf), "theta0 entries must be finite"),
    (lambda s: s.datasets[0].backgrounds[0].template.__setitem__(0, -1.0), "bkg_template"),
    (lambda s: s.datasets[0].backgrounds[0].template.__setitem__(1, np.nan), "bkg_template"),
    (lambda s: s.datasets[0].t.__setitem__(0, 1e39), "ds_t"),
    (lambda s: s.datasets[0].baseline.__setitem__(0, np.inf), "ds_weight / ds_baseline"),
    (lambda s: s.datasets[0].weight.__setitem__(0, np.inf), "ds_weight / ds_baseline"),
    (lambda s: setattr(s, "e_hi", np.inf), "energy grid"),
])
def test_description_numbers_must_be_finite(mutate, where):
    s = copy.deepcopy(synth.make_model("c0"))
    mutate(s)
    with pytest.raises(fitcore.FitError, match=where):
        fitcore.Model(s)


def test_every_synthetic_model_passes_the_host_checks():
    """The benchmark's and the tests' models pass every host check through both entry points:
    without a device the first error is the allocation's (with one, the model is created)."""
    for name in ["c0", "c0_tiny", "c1", "c2", "c1s", "c1_flux41"]:
        for remap in (0, 1):
            s = synth.make_model(name, remap=remap)
            rc, msg = _create(s.to_json())
            assert rc in (0, -4, -6), (name, remap, msg)
            try:
                fitcore.Model(s).close()
            except fitcore.FitError as e:
                assert "cudaMalloc" in str(e), (name, remap, str(e))


def _namespaced(cfg):
    """c0's configuration with its survival parameters in namespace "osc" and the rest in
    "det" (references rewritten to the full names)."""
    c = copy.deepcopy(cfg)
    osc = {e for e in c["oscillation"]["params"] if isinstance(e, str)}
    full = {p["name"]: ("osc." if p["name"] in osc else "det.") + p["name"] for p in c["parameters"]}
    c["parameters"] = [{"namespace": "osc", "parameters": [p for p in c["parameters"] if p["name"] in osc]},
                       {"namespace": "det", "parameters": [p for p in c["parameters"] if p["name"] not in osc]}]
    return json.dumps(c), full


def test_parameter_namespaces(cfg):
    text, full = _namespaced(cfg)
    assert _reject(text).count("unknown parameter")   # references still use the short names
    for short, long_ in full.items():
        text = text.replace(json.dumps(short), json.dumps(long_))
    text = text.replace('"name": "osc.', '"name": "').replace('"name": "det.', '"name": "')
    rc, msg = _create(text)
    assert rc in (0, -4, -6), msg
    c = json.loads(text)
    c["parameters"][0]["namespace"] = "a.b"
    assert "without '.'" in _reject(c)
    c = json.loads(text)
    c["parameters"][1]["parameters"].append(dict(c["parameters"][1]["parameters"][0]))
    assert 'duplicate name "det.' in _reject(c)


def _mapped_config(seed=3):
    """c1's configuration with the nine energy-scale coefficients constrained through a
    12-row linear map (each coefficient measured, plus three random combinations, with
    correlated errors of the coefficients' own sizes): Eq. 6 with b = A theta. Returns
    (config, A, b0, V, the coefficient names)."""
    spec = synth.make_model("c1")
    cfg = spec.to_config()
    esc = [f"a{k}[{d}]" for d in range(3) for k in range(3)]
    rng = np.random.default_rng(seed)
    A = np.vstack([np.eye(9), rng.standard_normal((3, 9))])
    w = np.array([0.01, 0.005, 0.001] * 3 + [0.005] * 3)
    Q = rng.standard_normal((12, 12))
    R = Q @ Q.T + 12 * np.eye(12)
    R /= np.sqrt(np.outer(np.diag(R), np.diag(R)))
    V = R * np.outer(w, w)
    b0 = A @ np.array([spec.theta0[spec.index(n)] for n in esc]) + 0.5 * w * rng.standard_normal(12)
    for p in cfg["parameters"]:
        if p["name"] in esc:
            p["sigma"] = 0.0
    cfg["covariances"].append({"params": esc, "map": A.tolist(), "mean": b0.tolist(), "cov": V.tolist()})
    return cfg, A, b0, V, esc


def test_linear_map_priors_are_checked_on_the_host():
    cfg, A, b0, V, esc = _mapped_config()
    rc, msg = _create(json.dumps(cfg))
    assert rc in (0, -4, -6), msg
    NON_SPD = -3
    c = copy.deepcopy(cfg)
    c["covariances"][-1]["map"] = np.zeros_like(A).tolist()
    rc, msg = _create(json.dumps(c))
    assert rc == NON_SPD and "does not fix every parameter" in msg
    c = copy.deepcopy(cfg)
    c["covariances"][-1]["cov"][0][0] = -1.0
    rc, msg = _create(json.dumps(c))
    assert rc == NON_SPD and ".cov: not positive definite" in msg
    c = copy.deepcopy(cfg)
    c["covariances"][-1].update(map=A[:5].tolist(), cov=V[:5, :5].tolist(), mean=b0[:5].tolist())
    assert "fewer rows than parameters" in _reject(c)
    c = copy.deepcopy(cfg)
    c["covariances"][-1]["mean"] = b0[:4].tolist()
    assert "one entry per map row" in _reject(c)


def _same(a, b, path=""):
    import dataclasses
    if dataclasses.is_dataclass(a):
        for f in dataclasses.fields(a):
            _same(getattr(a, f.name), getattr(b, f.name), path + "." + f.name)
    elif isinstance(a, (list, tuple)):
        assert len(a) == len(b), path
        for i, (x, y) in enumerate(zip(a, b)):
            _same(x, y, f"{path}[{i}]")
    elif isinstance(a, np.ndarray):
        assert np.array_equal(a, np.asarray(b)), path
        assert np.asarray(b).dtype.kind == a.dtype.kind, path
    else:
        assert a == b, (path, a, b)


@pytest.mark.parametrize("name", ["c0", "c0_tiny", "c1", "c2", "c1s", "c1_flux41"])
def test_description_round_trips_through_its_configuration(name):
    """ModelSpec.from_config(to_config()) is the description again, array for array, so the
    oracle can be built from any configuration the library reads."""
    for remap in (0, 1):
        s = synth.make_model(name, remap=remap)
        _same(s, synth.ModelSpec.from_config(s.to_json()), name)


def test_description_from_a_namespaced_configuration(cfg):
    text, full = _namespaced(cfg)
    for short, long_ in full.items():
        text = text.replace(json.dumps(short), json.dumps(long_))
    text = text.replace('"name": "osc.', '"name": "').replace('"name": "det.', '"name": "')
    s = synth.ModelSpec.from_config(text)
    assert s.param_names[:2] == ["osc.sin2_2th13", "osc.dm2_ee"]
    assert all(n.startswith(("osc.", "det.")) for n in s.param_names)
    assert s.osc_idx[0] == 0 and s.osc_idx[1] == 1
    cfg2, A, b0, V, esc = _mapped_config()
    s2 = synth.ModelSpec.from_config(cfg2)
    assert len(s2.map_priors) == 1
    ix, A2, b2, V2 = s2.map_priors[0]
    assert [s2.param_names[i] for i in ix] == esc
    assert np.array_equal(A2, A) and np.array_equal(b2, b0) and np.array_equal(V2, V)
    _same(s2, synth.ModelSpec.from_config(s2.to_json()), "mapped")
