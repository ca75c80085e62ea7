"""Learned warm start for the translation-invariant ADMM (an addition beyond the paper).

A WarmStart learns, for one instance family (fixed lattice and clusters, one model parameter:
the field h of the transverse-field Ising chain or the anisotropy Delta of the XXZ chain), the map
from the parameter to the solver's converged state, and starts new solves from its prediction:

  1. training states -- converged states for a grid of parameters, produced by the solver
     itself in one batch (ve_create_batch / ve_batch_iterate to a tight tolerance);
  2. compression -- the packed states are centred and projected on their leading principal
     directions (host SVD): K coefficients per state;
  3. regression -- a multilayer perceptron (ve_mlp_*: hand-written float32 kernels, trained on the
     GPU by Adam) maps the normalised parameter to the standardised coefficients;
  4. prediction -- coefficients -> state = mean + coefficients . directions, loaded with
     ve_set_state, after which ve_project_state_x projects X onto the PSD cone, so that the
     certified lower bound stays valid whatever the network predicts.

A prediction can leave small errors in the multipliers that the residual hardly shows but that
the certificate feels, so race_to_bound keeps the plain cold start beside it: a warm-started and
a cold copy of every instance advance in one batch, and each instance is done when either copy
certifies its target.
"""
import numpy as np

from . import ve


class WarmStart:
    def __init__(self, lattice, cluster, kind="tfim", n_components=16, hidden=256, layers=3,
                 seed=20210604):
        self.lattice, self.cluster, self.kind = tuple(lattice), tuple(cluster), kind
        self.K, self.hidden, self.layers, self.seed = n_components, hidden, layers, seed
        self.mlp = None

    def _ham(self, x):
        dim = len(self.lattice)
        return ve.ve_ham_tfim(dim, 1.0, x) if self.kind == "tfim" else ve.ve_ham_xxz(dim, 1.0, x)

    def _u(self, x):
        x = np.asarray(x, dtype=np.float64).reshape(-1, 1)
        return (2.0 * (x - self.lo) / (self.hi - self.lo) - 1.0).astype(np.float32)

    def training_states(self, xs, tol=1e-8, max_iter=60000, precision=ve.VE_PREC_MIXED):
        """Converged packed states for the parameters xs (one batch)."""
        inst = [(self.lattice, self.cluster, self._ham(x)) for x in xs]
        b = ve.ve_create_batch(inst, ve.ve_default_options(precision=precision))
        try:
            code, sts = ve.ve_batch_iterate(b, max_iter, tol)
            states = np.array([ve.ve_get_state(ve.ve_batch_handle(b, i)) for i in range(len(xs))])
        finally:
            ve.ve_batch_destroy(b)
        return states, sts

    def fit(self, xs, states, train_steps=4000, lr=1e-3):
        """Compress `states` (one row per parameter in xs) and train the network; returns the
        final training loss (standardised coefficient units)."""
        xs = np.asarray(xs, dtype=np.float64)
        self.lo, self.hi = float(xs.min()), float(xs.max())
        self.mean = states.mean(axis=0)
        centred = states - self.mean
        _, sv, vt = np.linalg.svd(centred, full_matrices=False)
        K = min(self.K, vt.shape[0])
        self.basis = vt[:K]
        coeff = centred @ self.basis.T
        self.cscale = coeff.std(axis=0) + 1e-30
        self.explained = float(np.sum(sv[:K] ** 2) / max(1e-300, np.sum(sv ** 2)))
        target = (coeff / self.cscale).astype(np.float32)
        if self.mlp:
            ve.ve_mlp_destroy(self.mlp)
        self.mlp = ve.ve_mlp_create(1, self.hidden, self.layers, K, self.seed)
        return ve.ve_mlp_train(self.mlp, self._u(xs), target, train_steps, lr)

    def predict_state(self, x):
        c = ve.ve_mlp_predict(self.mlp, self._u([x]), self.basis.shape[0])[0].astype(np.float64)
        return self.mean + (c * self.cscale) @ self.basis

    def apply(self, handle, x):
        """Load the predicted state for parameter x into `handle` and make its X PSD."""
        ve.ve_set_state(handle, self.predict_state(x))
        ve.ve_project_state_x(handle)

    def close(self):
        if self.mlp:
            ve.ve_mlp_destroy(self.mlp)
            self.mlp = None


def race_to_bound(lattice, cluster, kind, params, targets, warm, chunk=50, max_sweeps=40000,
                  precision=ve.VE_PREC_MIXED):
    """Certify, for every parameter in `params`, a lower bound per spin >= the matching entry of
    `targets`.  A warm-started (from `warm`, a fitted WarmStart of this family) and a cold copy
    of each instance run side by side in one batch; the bound of every copy is certified every
    `chunk` sweeps.  Returns one dict per instance: sweeps when first certified (None if not
    within max_sweeps), the copy that got there ('warm' or 'cold') and its bound."""
    dim = len(lattice)
    ham = (lambda x: ve.ve_ham_tfim(dim, 1.0, x)) if kind == "tfim" else (
        lambda x: ve.ve_ham_xxz(dim, 1.0, x))
    n = len(params)
    inst = [(tuple(lattice), tuple(cluster), ham(x)) for x in params] * 2
    b = ve.ve_create_batch(inst, ve.ve_default_options(precision=precision))
    res = [{"sweeps": None, "copy": None, "bound_per_spin": None} for _ in range(n)]
    try:
        for i, x in enumerate(params):
            warm.apply(ve.ve_batch_handle(b, i), x)
        while True:
            _, sts = ve.ve_batch_iterate(b, chunk, 1e-13)
            sweeps = max(s.iter for s in sts)
            certs = ve.ve_batch_bound(b)
            for i in range(n):
                if res[i]["sweeps"] is not None:
                    continue
                for copy, c in (("warm", certs[i]), ("cold", certs[n + i])):
                    if c.bound_per_spin >= targets[i]:
                        res[i] = {"sweeps": sweeps, "copy": copy, "bound_per_spin": c.bound_per_spin}
                        break
            if all(r["sweeps"] is not None for r in res) or sweeps >= max_sweeps:
                return res
    finally:
        ve.ve_batch_destroy(b)
