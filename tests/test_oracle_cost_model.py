"""Pins of the cost-model network oracle (oracle/cost_model.py).

* backward against FP64 central differences of the loss;
* forward special cases whose value is known without the network: all
  weights zero gives the output bias; one open path through one hidden unit
  gives tanh of its bias times the output weight;
* the first Adam step from zero moments moves every weight by lr times the
  sign of its gradient (the bias corrections cancel the (1 - beta) factors)."""
import numpy as np

from oracle import cost_model as C


def _batch(rng, b=37):
    x = np.stack([rng.uniform(0, 11, b), rng.uniform(0, 11, b), rng.uniform(2, 5, b),
                  rng.integers(2, 16, b)], axis=1)
    t = rng.normal(0, 2, (b, 2))
    m = (rng.random((b, 2)) < 0.6).astype(np.float64)
    m[0] = 1.0
    return x, t, m


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.4, C.NPARAM)
    x, t, m = _batch(rng)
    _, g = C.grad(theta, x, t, m)
    idx = rng.choice(C.NPARAM, 300, replace=False)
    idx = np.concatenate([idx, np.arange(C.NPARAM - 130, C.NPARAM)])  # all of W3, b3
    h = 1e-6
    fd = np.empty(len(idx))
    for k, i in enumerate(idx):
        e = np.zeros(C.NPARAM)
        e[i] = h
        fd[k] = (C.loss(theta + e, x, t, m) - C.loss(theta - e, x, t, m)) / (2 * h)
    assert np.max(np.abs(fd - g[idx])) <= 1e-7 * max(1.0, np.max(np.abs(g[idx])))


def test_forward_special_cases():
    rng = np.random.default_rng(1)
    x, _, _ = _batch(rng, 9)
    P = {name: np.zeros(shp) for name, shp in C.SHAPES}
    P["b3"] = np.array([0.25, -1.5])
    y, _ = C.forward(C.pack(P), x)
    assert np.array_equal(y, np.tile(P["b3"], (9, 1)))
    # one path: hidden unit 7 of layer 2 fixed at tanh(b2[7]) = 0.5
    P["b2"][7] = np.arctanh(0.5)
    P["W3"][1, 7] = 3.0
    y, _ = C.forward(C.pack(P), x)
    assert np.allclose(y[:, 0], 0.25, rtol=0, atol=1e-15)
    assert np.allclose(y[:, 1], -1.5 + 3.0 * 0.5, rtol=0, atol=1e-14)


def test_first_adam_step_is_sign_step():
    rng = np.random.default_rng(2)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    w1, mom, vel = C.adam_step(w, np.zeros(50), np.zeros(50), g, 1, 1e-3, eps=0.0)
    assert np.allclose(w1 - w, -1e-3 * np.sign(g), rtol=1e-12, atol=0)
    assert np.allclose(mom, 0.1 * g) and np.allclose(vel, 0.001 * g * g)


def test_training_reduces_loss_on_a_smooth_target():
    rng = np.random.default_rng(3)
    x, _, m = _batch(rng, 256)
    m[:] = 1.0
    t = np.stack([0.3 * x[:, 0] + 0.5 * x[:, 1] - 3.0, np.log(x[:, 3] ** 2)], axis=1)
    w = rng.normal(0, 0.2, C.NPARAM)
    mom, vel = np.zeros_like(w), np.zeros_like(w)
    l0 = C.loss(w, x, t, m)
    for s in range(1, 301):
        _, g = C.grad(w, x, t, m)
        w, mom, vel = C.adam_step(w, mom, vel, g, s, 1e-2)
    assert C.loss(w, x, t, m) < 0.05 * l0


def test_fp16_rounding_is_binary16():
    v = np.array([1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 65504.0, 1e-8])
    r = C.to_fp16(v)
    assert r[0] == 1.0 and r[1] == 1.0 + 2.0 ** -9 and r[2] == 65504.0 and r[3] == 0.0
