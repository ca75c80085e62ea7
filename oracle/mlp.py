"""CPU float64 multilayer perceptron: the reference for the GPU warm-start network's forward
pass and gradients.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Same network and parameter layout as the
library's ve_mlp: a_0 = x, a_l = tanh(W_l a_{l-1} + b_l) for the hidden layers, y = W_out a + b_out;
loss = mean over samples and outputs of (y - t)^2 / 2; parameters stored layer by layer, W
(outputs x inputs, row-major) then b.  Backpropagation is the chain rule written out layer by
layer; it is pinned against central finite differences in tests/test_oracle_pins.py.
"""
import numpy as np


def layer_shapes(n_in, n_hidden, n_layers, n_out):
    dims = [n_in] + [n_hidden] * n_layers + [n_out]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def unpack(params, shapes):
    out, off = [], 0
    for (o, i) in shapes:
        W = params[off:off + o * i].reshape(o, i)
        off += o * i
        b = params[off:off + o]
        off += o
        out.append((W, b))
    assert off == params.size
    return out


def forward(params, shapes, x):
    layers = unpack(np.asarray(params, dtype=np.float64), shapes)
    acts = [np.asarray(x, dtype=np.float64)]
    for l, (W, b) in enumerate(layers):
        z = acts[-1] @ W.T + b
        acts.append(np.tanh(z) if l < len(layers) - 1 else z)
    return acts


def loss_grad(params, shapes, x, t):
    """(loss, gradient with respect to the flat parameter vector)"""
    t = np.asarray(t, dtype=np.float64)
    acts = forward(params, shapes, x)
    layers = unpack(np.asarray(params, dtype=np.float64), shapes)
    y = acts[-1]
    r = y - t
    loss = 0.5 * np.mean(r * r)
    dz = r / r.size
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = (dz.T @ acts[l], dz.sum(axis=0))
        if l > 0:
            dz = (dz @ W) * (1.0 - acts[l] ** 2)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat
