"""Learned warm start: collect training pairs from the method's own
demagnetisation-curve trajectories, train the network with the library's
tensor-core kernels, and run a curve with the warm start applied before
every minimisation (Algorithm 4 still runs to t1-t3 from the corrected
state).

Training pairs: at the converged state of field step k, the features for the
step to field k+1 (mm_warmstart_features) and the targets
((m_{k+1} - m_k), (phi_{k+1} - phi_k)) / |dh| on the magnetic nodes, where
|dh| is the norm of the field increment in internal units
(mm_warmstart_targets).  The network standardises its inputs itself (FP32,
before the BF16 first layer; features such as m_z = 0.999 +- 0.001 would
lose their signal if the standardisation were folded into BF16 weights);
the statistics (mm_mlp_fit_input_norm) and the target scales
(mm_mlp_fit_target_scales), which become the scale_m / scale_phi arguments
of mm_warmstart_apply, are computed by the library.  This module only
moves tensors: it concatenates the steps' arrays and draws the
mini-batches.
"""
from .api import Params, warmstart_features, warmstart_apply


def collect(mag, mlp, m0, fields, n_mag, params=None, max_step_change=0.2):
    """Run the curve on `mag` from m0 and return device tensors (X, T, nli):
    features and targets (mm_warmstart_targets) of every field step.  Field
    steps on which some node turned by more than max_step_change
    (irreversible switching) are left out: the network is to learn the
    reversible response that keeps the state in its basin, not to jump."""
    import torch
    prm = params or Params()
    mag.set_magnetization(m0)
    mag.set_field(fields[0])
    nli = mag.minimize(prm)["nli"]
    Xs, Ts = [], []
    for k in range(len(fields) - 1):
        X = warmstart_features(mag, fields[k + 1], n_mag)
        mag.set_field(fields[k + 1])
        nli += mag.minimize(prm)["nli"]
        X1 = warmstart_features(mag, fields[k + 1], n_mag)
        T, dh, change = mlp.step_targets(X, X1)
        if T is None or change > max_step_change:
            continue
        Xs.append(X)
        Ts.append(T)
    return torch.cat(Xs), torch.cat(Ts), nli


def train(mlp, X, T, steps=2000, batch=16384, lr=2e-3, seed=0, log_every=0):
    """Set the network's input standardisation from X and the target scales
    from T (both computed by the library), then train with Adam on random
    mini-batches of the standardised targets.  Returns (scale_m, scale_phi,
    losses)."""
    import torch
    mlp.fit_input_norm(X)
    Tn, s_m, s_p = mlp.fit_target_scales(T)
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    n = X.shape[0]
    losses = []
    for it in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), device=X.device, generator=g)
        xb = X[idx].contiguous()
        tb = Tn[idx].contiguous()
        want = bool(log_every) and (it % log_every == 0 or it == steps - 1)
        loss = mlp.train_step(xb, tb, lr, want_loss=want)
        if want:
            losses.append((it, loss))
    return s_m, s_p, losses


def curve(mag, m0, fields, params=None, mlp=None, scales=None, max_change=0.02):
    """Demagnetisation curve; with `mlp`, the warm start is applied before
    every field step after the first.  Returns (stats per step, total nli)."""
    prm = params or Params()
    mag.set_magnetization(m0)
    out = []
    for k, b in enumerate(fields):
        if mlp is not None and k > 0:
            warmstart_apply(mag, mlp, b, scales[0], scales[1], max_change)
        mag.set_field(b)
        out.append(mag.minimize(prm))
    return out, sum(s["nli"] for s in out)
