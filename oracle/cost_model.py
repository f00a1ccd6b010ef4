"""FP64 numpy oracle of the learned cost model's network: forward pass, loss,
backward pass and one Adam step.

TEST INFRASTRUCTURE ONLY: the library never imports this module.  It shares no
code with the CUDA kernels that train and evaluate the network on the GPU.

The network (a 3-layer perceptron, hidden width 64, FP16 parameters) predicts
the cost of one cell pair for the two interaction types the hybrid traversal
chooses between (section "A new hybrid treecode-FMM with auto-tuning": the
kernels are timed on artificial data and the cheapest is selected during the
traversal; here a network fitted to those timings stands in for the table of
timings):

    u   = (x - MU) / SD                 x = (log2 n_t, log2 n_s, sep, p)
    h1  = tanh(W1 u + b1)               W1: 64 x 4
    h2  = tanh(W2 h1 + b2)              W2: 64 x 64
    y   = W3 h2 + b3                    W3: 2 x 64,  y = (ln t_P2P, ln t_M2L)

with t the time per pair in nanoseconds and sep the separation-to-size ratio
R / (r_t + r_s).  The loss over a batch with a mask m (1 where the sample has a
measured value of that output) is

    loss = sum_{s,k} m_sk (y_sk - t_sk)^2 / sum_{s,k} m_sk .

Parameters are one flat vector in the order W1 (row-major), b1, W2, b2, W3, b3.
Adam: Kingma & Ba, "Adam: a method for stochastic optimization" (2015), with
bias-corrected moments.
"""
from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 4, 64, 2
MU = np.array([5.0, 5.0, 3.0, 8.0])
SD = np.array([4.0, 4.0, 1.5, 4.0])
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
          ("W3", (NOUT, NH)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (NPARAM,)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], np.float64).reshape(-1) for name, _ in SHAPES])


def forward(theta, x):
    """Predictions y [B, 2] and the activations needed by backward."""
    P = unpack(theta)
    u = (np.asarray(x, np.float64) - MU) / SD
    h1 = np.tanh(u @ P["W1"].T + P["b1"])
    h2 = np.tanh(h1 @ P["W2"].T + P["b2"])
    y = h2 @ P["W3"].T + P["b3"]
    return y, (u, h1, h2)


def loss(theta, x, t, m):
    y, _ = forward(theta, x)
    m = np.asarray(m, np.float64)
    return float(np.sum(m * (y - t) ** 2) / max(np.sum(m), 1.0))


def grad(theta, x, t, m):
    """(loss, d loss / d theta) by the chain rule through the three layers."""
    P = unpack(theta)
    y, (u, h1, h2) = forward(theta, x)
    m = np.asarray(m, np.float64)
    cnt = max(np.sum(m), 1.0)
    dy = 2.0 * m * (y - t) / cnt                 # [B, 2]
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dz2 = (dy @ P["W3"]) * (1.0 - h2 ** 2)       # [B, 64]
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * (1.0 - h1 ** 2)
    g["W1"] = dz1.T @ u
    g["b1"] = dz1.sum(0)
    return float(np.sum(m * (y - t) ** 2) / cnt), pack(g)


def adam_step(w, mom, vel, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of the FP64 master weights; returns (w, mom, vel)."""
    mom = beta1 * mom + (1.0 - beta1) * g
    vel = beta2 * vel + (1.0 - beta2) * g * g
    mh = mom / (1.0 - beta1 ** step)
    vh = vel / (1.0 - beta2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), mom, vel


def to_fp16(theta):
    """Parameters as the network stores them (IEEE binary16, round to nearest)."""
    return np.asarray(theta, np.float64).astype(np.float16).astype(np.float64)
