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


class StencilWarmStart:
    """A warm start that transfers across lattice sizes: an MLP maps the model parameter (the
    field h of the transverse-field Ising model, or the XXZ anisotropy Delta; J = 1) to the blocks
    X_{0,delta} of the converged dual matrix at the offsets of the unit stencil -- delta = 0 and
    one step along each axis (the opposite steps are their transposes, X_{0,-delta} =
    X_{0,delta}^T).  Those blocks are lattice-size independent up to the correlation length, so
    a network trained on solves of a small lattice starts a larger one: every variable at its
    cold initial value except X, whose stencil blocks come from the prediction (all other blocks
    zero), projected onto the PSD cone (ve_project_state_x) so the certificate stays valid.

    Where it helps: on the 2-D transverse-field Ising model at h = 3 (paramagnetic, gapped) the
    oracle needs 6120 instead of 9640 sweeps to the 1e-6 residual on a 12 x 12 lattice started
    from the 8 x 8 lattice's converged stencil.  On the XXZ model it does not: at Delta = 1.5 the
    same transfer costs 9310 sweeps against 7480 cold, and at Delta = 0.5 even the lattice's own
    converged X (stencil or whole) costs 1480 against 1080 -- there the dual matrix alone is the
    wrong thing to carry over, and the plain cold start remains the reference."""

    def __init__(self, cluster, dim, kind="tfim", hidden=256, layers=3, seed=20210604):
        self.cluster, self.dim, self.kind = tuple(cluster), int(dim), kind
        self.hidden, self.layers, self.seed = hidden, layers, seed
        self.mlp = None

    def _ham(self, x):
        return ve.ve_ham_tfim(self.dim, 1.0, x) if self.kind == "tfim" else ve.ve_ham_xxz(self.dim, 1.0, x)

    def _u(self, x):
        x = np.asarray(x, dtype=np.float64).reshape(-1, 1)
        return (2.0 * (x - self.lo) / (self.hi - self.lo) - 1.0).astype(np.float32)

    def _layout(self, lattice, h):
        """(D, offset of X in the packed state, clusters per axis) of a handle on `lattice`."""
        N, m, D = ve.ve_dims(h)
        P = N - 1
        M = [lattice[a] // self.cluster[a] for a in range(self.dim)]
        return D, m * m + 2 * P * D * D + 2 * P * m * m, M

    def _offsets(self, M):
        """Linear indices of the stencil offsets: 0, then +e_a and -e_a for every axis a."""
        def lin(v):
            idx = 0
            for a in range(self.dim):
                idx = idx * M[a] + (v[a] % M[a])
            return idx
        steps = []
        for a in range(self.dim):
            e = [0] * self.dim
            e[a] = 1
            steps.append((lin(e), lin([-c for c in e])))
        return lin([0] * self.dim), steps

    def stencil(self, lattice, h, state):
        """The stencil blocks of a packed state: X_{0,0} and X_{0,+e_a} for each axis, flattened."""
        D, xo, M = self._layout(lattice, h)
        z, steps = self._offsets(M)
        blocks = [state[xo + z * D * D: xo + (z + 1) * D * D]]
        for plus, _ in steps:
            blocks.append(state[xo + plus * D * D: xo + (plus + 1) * D * D])
        return np.concatenate(blocks)

    def train(self, lattice, xs, tol=1e-6, max_iter=40000, precision=ve.VE_PREC_FP64,
              train_steps=3000, lr=1e-3):
        """Solve `lattice` for every parameter in xs (one batch), take the stencil blocks of the
        converged X and fit the network; returns the final training loss."""
        assert all(lattice[a] // self.cluster[a] >= 3 for a in range(self.dim)), \
            "the stencil needs at least 3 clusters along every axis"
        inst = [(tuple(lattice), self.cluster, self._ham(x)) for x in xs]
        b = ve.ve_create_batch(inst, ve.ve_default_options(precision=precision))
        try:
            ve.ve_batch_iterate(b, max_iter, tol)
            feats = np.array([self.stencil(lattice, ve.ve_batch_handle(b, i),
                                           ve.ve_get_state(ve.ve_batch_handle(b, i)))
                              for i in range(len(xs))])
        finally:
            ve.ve_batch_destroy(b)
        xs = np.asarray(xs, dtype=np.float64)
        self.lo, self.hi = float(xs.min()), float(xs.max())
        self.fmean = feats.mean(axis=0)
        self.fscale = feats.std(axis=0) + 1e-12
        target = ((feats - self.fmean) / self.fscale).astype(np.float32)
        if self.mlp:
            ve.ve_mlp_destroy(self.mlp)
        self.mlp = ve.ve_mlp_create(1, self.hidden, self.layers, target.shape[1], self.seed)
        return ve.ve_mlp_train(self.mlp, self._u(xs), target, train_steps, lr)

    def predict(self, x):
        y = ve.ve_mlp_predict(self.mlp, self._u([x]), self.fmean.size)[0].astype(np.float64)
        return self.fmean + y * self.fscale

    def apply(self, handle, lattice, x):
        """Start `handle` (a fresh handle on `lattice`, any size with >= 3 clusters per axis)
        from the cold state with the predicted stencil blocks of X, made PSD."""
        D, xo, M = self._layout(lattice, handle)
        z, steps = self._offsets(M)
        state = ve.ve_get_state(handle)
        f = self.predict(x).reshape(-1, D, D)
        X = state[xo:].reshape(-1, D, D)
        X[:] = 0.0
        X[z] = 0.5 * (f[0] + f[0].T)
        for k, (plus, minus) in enumerate(steps):
            X[plus] = f[1 + k]
            X[minus] = f[1 + k].T
        ve.ve_set_state(handle, state)
        ve.ve_project_state_x(handle)

    def close(self):
        if self.mlp:
            ve.ve_mlp_destroy(self.mlp)
            self.mlp = None
