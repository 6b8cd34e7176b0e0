"""CPU reference of the warm-start network (an extension of the method; the paper
has no learned component): a per-node multilayer perceptron
16 -> 128 -> 128 -> 128 -> 4 with ReLU, trained by mean squared error.

The GPU kernels compute in BF16 with FP32 accumulation.  This reference
rounds to BF16 (round to nearest even) at the same points -- the input
features, the weights and every hidden activation before it is multiplied --
and computes everything else in FP64, so the two agree up to FP32
accumulation order and the occasional tie in a BF16 rounding.

Backward pass (written out from the chain rule, per layer l with
z_l = a_{l-1} W_l^T + b_l, a_l = relu(z_l)):
  dL/dy = 2 (y - t) / (N * n_out)
  dW_l = dz_l^T a_{l-1},  db_l = sum over rows of dz_l,
  da_{l-1} = dz_l W_l,    dz_{l-1} = da_{l-1} * [z_{l-1} > 0].
The hidden activations a_{l-1} used for dW_l are the BF16-rounded ones.

Pins (tests/test_oracle_mlp.py): central differences of the loss (with the
BF16 rounding switched off, so the loss is smooth in the weights), a linear
network's closed-form gradient, and the BF16 rounding against exact values.
"""
import numpy as np

SIZES = (16, 128, 128, 128, 4)


def bf16(x):
    """Round FP32/FP64 values to the nearest BF16 value (ties to even),
    returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out[nan] = np.nan
    return out


def init_params(seed, sizes=SIZES):
    """He-uniform weights W_l [out, in] and zero biases (FP32 values)."""
    rng = np.random.default_rng(seed)
    params = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / n_in)
        W = rng.uniform(-lim, lim, size=(n_out, n_in)).astype(np.float32).astype(np.float64)
        b = np.zeros(n_out)
        params.append((W, b))
    return params


def forward(params, X, round_bf16=True):
    """Returns the output and the per-layer (input activation, pre-activation)."""
    rnd = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    a = rnd(X)
    cache = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = a @ rnd(W).T + b
        cache.append((a, z))
        if l < L - 1:
            a = rnd(np.maximum(z, 0.0))
        else:
            a = z
    return a, cache


def loss_and_grads(params, X, T, round_bf16=True):
    """Mean squared error over all outputs and its gradients
    [(dW_l, db_l), ...]."""
    rnd = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    Y, cache = forward(params, X, round_bf16)
    N, n_out = Y.shape
    diff = Y - T
    loss = float(np.sum(diff * diff) / (N * n_out))
    dz = 2.0 * diff / (N * n_out)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        a_prev, z = cache[l]
        W, b = params[l]
        grads[l] = (dz.T @ a_prev, dz.sum(axis=0))
        if l > 0:
            da = dz @ rnd(W)
            z_prev = cache[l - 1][1]
            dz = da * (z_prev > 0.0)
    return loss, grads
