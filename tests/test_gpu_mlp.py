"""Warm-start network on the tensor cores (bf16 operands, FP32 accumulation) against the FP64
reference network, plus the feature and start-point kernels of the warm start.

Tolerance: ||y - y_ref|| / ||y_ref|| <= 1e-2 for outputs and for each layer's gradients. Every
operand (inputs, weights, activations, the back-propagated error) is rounded to bf16 (8
significant bits, relative error <= 2^-9 each); sums of many such products keep the relative
error of a layer at the 2^-9 level, a handful of layers well inside 1e-2.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as ref_mlp
from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _weights(net):
    return [net.get_layer(l)[:2] for l in range(net.n_layers)]


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dims,B", [((70, 96, 2, 12), 300), ((438, 512, 3, 12), 1000),
                                    ((5, 16, 0, 3), 7)])
def test_forward_matches_reference(dims, B):
    net = fitcore.Mlp(*dims, seed=5)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((B, dims[0])).astype(np.float32)
    y = torch.zeros((B, dims[3]), dtype=torch.float32, device="cuda")
    net.forward(B, torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    ref, _, _ = ref_mlp.forward(_weights(net), x)
    assert _rel(y.cpu().numpy(), ref) <= 1e-2


def test_gradients_loss_and_adamw_step():
    net = fitcore.Mlp(70, 96, 2, 12, seed=6)
    rng = np.random.default_rng(2)
    B = 300
    x = rng.standard_normal((B, 70)).astype(np.float32)
    t = rng.standard_normal((B, 12)).astype(np.float32)
    w0 = _weights(net)
    loss = np.zeros(1)
    lr, wd = 1e-3, 0.01
    net.train_step(B, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), lr, wd, loss)
    torch.cuda.synchronize()
    ref_loss, ref_grads = ref_mlp.loss_and_grads(w0, x, t)
    assert abs(loss[0] - ref_loss) <= 1e-2 * ref_loss
    for l in range(net.n_layers):
        w1, b1, gw, gb = net.get_layer(l)
        assert _rel(gw, ref_grads[l][0]) <= 1e-2, l
        assert _rel(gb, ref_grads[l][1]) <= 1e-2, l
        # AdamW from the device's own gradient: the first step is exact up to FP32 rounding
        wr, _, _ = ref_mlp.adamw_step(w0[l][0].astype(np.float64), gw.astype(np.float64),
                                      0.0, 0.0, 1, lr, wd)
        br, _, _ = ref_mlp.adamw_step(w0[l][1].astype(np.float64), gb.astype(np.float64),
                                      0.0, 0.0, 1, lr, wd, decay=False)
        np.testing.assert_allclose(w1, wr, rtol=0, atol=lr * 1e-4 + 1e-6 * np.abs(wr).max())
        np.testing.assert_allclose(b1, br, rtol=0, atol=lr * 1e-4 + 1e-6 * np.abs(br).max())


def test_training_reduces_loss_on_a_teacher():
    net = fitcore.Mlp(40, 64, 2, 6, seed=7)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 6)) / np.sqrt(40)
    B = 512
    losses = []
    buf = np.zeros(1)
    for it in range(300):
        x = rng.standard_normal((B, 40)).astype(np.float32)
        t = np.tanh(x @ A).astype(np.float32)
        net.train_step(B, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), 2e-3, 0.0, buf)
        losses.append(buf[0])
    assert np.mean(losses[-20:]) < 0.1 * np.mean(losses[:5])


def test_set_layer_round_trip():
    net = fitcore.Mlp(9, 16, 1, 4, seed=8)
    rng = np.random.default_rng(4)
    w = rng.standard_normal((16, 9)).astype(np.float32)
    b = rng.standard_normal(16).astype(np.float32)
    net.set_layer(0, w, b)
    w2, b2, _, _ = net.get_layer(0)
    np.testing.assert_array_equal(w, w2)
    np.testing.assert_array_equal(b, b2)
    x = rng.standard_normal((33, 9)).astype(np.float32)
    y = torch.zeros((33, 4), dtype=torch.float32, device="cuda")
    net.forward(33, torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    assert _rel(y.cpu().numpy(), ref_mlp.forward(_weights(net), x)[0]) <= 1e-2


@pytest.mark.parametrize("name,slot0,onehot", [("c1", 0, 114), ("c0", 10, -1)])
def test_features_and_start_points(name, slot0, onehot):
    spec = synth.make_model(name)
    om = oracle.OracleModel(spec)
    gm = fitcore.Model(spec)
    nbar = om.expected(spec.theta0)
    B, n_in = 37, 438
    data = np.stack([synth.poisson_data(nbar, 100 + b) for b in range(B)]).astype(np.float32)
    dd = torch.from_numpy(data).cuda()
    x = torch.zeros((B, n_in), dtype=torch.float32, device="cuda")
    fitcore.fit_warmstart_features(gm, B, dd, None, n_in, slot0, onehot, x)
    torch.cuda.synchronize()
    ref = np.zeros((B, n_in))
    ref[:, slot0:slot0 + gm.n_data] = np.log1p(data) / np.log1p(nbar) - 1.0
    if onehot >= 0:
        ref[:, onehot] = 1.0
    np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=0, atol=2e-6)
    # dataset masks: the bins of a left-out dataset read 0
    n_ds = len(spec.datasets)
    masks = np.array([(1 << n_ds) - 1 if b % 2 else 1 for b in range(B)], np.uint32)
    fitcore.fit_warmstart_features(gm, B, dd, torch.from_numpy(masks.view(np.int32)).cuda(),
                                   n_in, slot0, onehot, x)
    torch.cuda.synchronize()
    off = 0
    for d, ds in enumerate(spec.datasets):
        n = spec.detectors[ds.det].n_reco
        keep = (masks >> d) & 1
        ref[:, slot0 + off:slot0 + off + n] *= keep[:, None]
        off += n
    np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=0, atol=2e-6)
    # start points: the linearised start, plus y_t * scale_t on the target parameters
    net = fitcore.Mlp(n_in, 64, 1, 12, seed=9)
    idx = np.arange(3)
    scl = np.array([0.01, 0.02, 0.03])
    th = torch.zeros((B, gm.n_params), dtype=torch.float64, device="cuda")
    base = torch.zeros_like(th)
    fitcore.fit_warmstart_features(gm, B, dd, None, n_in, slot0, onehot, x)
    fitcore.fit_warmstart_predict(net, gm, B, dd, None, slot0, onehot, idx, scl, th)
    fitcore.fit_linear_start(gm, B, dd, None, base)
    y = torch.zeros((B, 12), dtype=torch.float32, device="cuda")
    net.forward(B, x, y)
    torch.cuda.synchronize()
    expect = base.cpu().numpy().copy()
    expect[:, idx] += y.cpu().numpy()[:, :3].astype(np.float64) * scl
    np.testing.assert_allclose(th.cpu().numpy(), expect, rtol=1e-12, atol=1e-12)
