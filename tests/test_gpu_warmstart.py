"""The learned warm start: the GPU network against the CPU float64 reference, and the warm start
against cold starts on held-out parameters."""
import numpy as np
import pytest

import __graft_entry__
from oracle import mlp
from oracle import models as mo

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ve():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    __graft_entry__.build()
    from paper_2106_02682_gb300 import ve as mod
    return mod


@pytest.mark.parametrize("n_in,hidden,layers,n_out,n", [(1, 256, 3, 16, 37), (3, 40, 2, 5, 9)])
def test_gpu_network_matches_the_reference(ve, n_in, hidden, layers, n_out, n):
    rng = np.random.default_rng(7)
    m = ve.ve_mlp_create(n_in, hidden, layers, n_out, 11)
    try:
        shapes = mlp.layer_shapes(n_in, hidden, layers, n_out)
        assert ve.ve_mlp_num_params(m) == sum(o * i + o for o, i in shapes)
        p = ve.ve_mlp_get_params(m).astype(np.float64)
        x = rng.normal(size=(n, n_in)).astype(np.float32)
        t = rng.normal(size=(n, n_out)).astype(np.float32)
        loss, g = ve.ve_mlp_loss_grad(m, x, t)
        rloss, rg = mlp.loss_grad(p, shapes, x, t)
        assert abs(loss - rloss) <= 1e-5 * max(1.0, abs(rloss))
        assert np.max(np.abs(g - rg)) <= 1e-4 * np.max(np.abs(rg))
        y = ve.ve_mlp_predict(m, x, n_out)
        np.testing.assert_allclose(y, mlp.forward(p, shapes, x)[-1], atol=2e-5, rtol=1e-4)
        # training lowers the loss
        assert ve.ve_mlp_train(m, x, t, 1500, 1e-3) < 0.5 * rloss
    finally:
        ve.ve_mlp_destroy(m)


def test_training_is_reproducible_bit_for_bit(ve):
    """Two networks from the same seed trained on the same data end with identical parameters
    and loss: the training reductions have a fixed order (no atomics)."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=(24, 1)).astype(np.float32)
    t = rng.normal(size=(24, 8)).astype(np.float32)
    out = []
    for _ in range(2):
        m = ve.ve_mlp_create(1, 64, 3, 8, 5)
        try:
            loss = ve.ve_mlp_train(m, x, t, 300, 1e-3)
            out.append((loss, ve.ve_mlp_get_params(m).copy()))
        finally:
            ve.ve_mlp_destroy(m)
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])


LATTICE, CLUSTER = (40,), (2,)


@pytest.fixture(scope="module")
def fitted(ve):
    from paper_2106_02682_gb300.warmstart import WarmStart
    ws = WarmStart(LATTICE, CLUSTER, "tfim", n_components=12)
    xs = np.linspace(0.5, 1.5, 11)
    states, _ = ws.training_states(xs, tol=1e-8, max_iter=40000)
    loss = ws.fit(xs, states, train_steps=3000)
    yield ws, loss
    ws.close()


def test_warm_start_beats_cold_start_on_held_out_fields(ve, fitted):
    ws, loss = fitted
    lattice, cluster = LATTICE, CLUSTER
    assert loss < 1e-2
    opt = ve.ve_default_options(precision=1)
    cold_total = warm_total = 0
    for h in (0.65, 0.95, 1.25):
        hc = ve.ve_create(lattice, cluster, ve.ve_ham_tfim(1, 1.0, h), opt)
        hw = ve.ve_create(lattice, cluster, ve.ve_ham_tfim(1, 1.0, h), opt)
        try:
            _, sc = ve.ve_iterate(hc, 40000, 1e-6)
            ws.apply(hw, h)
            assert ve.ve_bound(hw).x_min_eig > -1e-9          # X is PSD after the projection
            _, sw = ve.ve_iterate(hw, 40000, 1e-6)
            cold_total += sc.iter
            warm_total += sw.iter
            bound = ve.ve_bound(hw).bound_per_spin
            assert bound <= mo.tfim_chain_jw_energy(40, 1.0, h) / 40     # still a lower bound
        finally:
            ve.ve_destroy(hc)
            ve.ve_destroy(hw)
    assert warm_total < 0.7 * cold_total, (warm_total, cold_total)


def test_race_certifies_every_target_no_later_than_the_cold_start(ve, fitted):
    """Warm and cold copies raced in one batch: every instance reaches its target (the float64
    bound at the residual 1e-6, less 1e-6), never later than a cold mixed solve checked on the
    same 50-sweep grid, and every certified bound stays below the exact energy."""
    from paper_2106_02682_gb300.warmstart import race_to_bound
    ws, _ = fitted
    fields = [0.65, 0.95, 1.25]
    targets, cold = [], []
    for h in fields:
        hf = ve.ve_create(LATTICE, CLUSTER, ve.ve_ham_tfim(1, 1.0, h), ve.ve_default_options(precision=0))
        hc = ve.ve_create(LATTICE, CLUSTER, ve.ve_ham_tfim(1, 1.0, h), ve.ve_default_options(precision=1))
        try:
            ve.ve_iterate(hf, 40000, 1e-6)
            targets.append(ve.ve_bound(hf).bound_per_spin - 1e-6)
            while True:
                _, st = ve.ve_iterate(hc, 50, 1e-13)
                if ve.ve_bound(hc).bound_per_spin >= targets[-1] or st.iter >= 40000:
                    cold.append(st.iter)
                    break
        finally:
            ve.ve_destroy(hf)
            ve.ve_destroy(hc)
    race = race_to_bound(LATTICE, CLUSTER, "tfim", fields, targets, ws, chunk=50, max_sweeps=40000)
    for h, t, c, r in zip(fields, targets, cold, race):
        assert r["sweeps"] is not None and r["sweeps"] <= c, (h, r, c)
        assert t <= r["bound_per_spin"] <= mo.tfim_chain_jw_energy(40, 1.0, h) / 40


def test_stencil_warm_start_transfers_to_a_larger_lattice(ve):
    """The lattice-size-independent warm start: a network trained on 8 x 8 solves of the 2-D
    transverse-field Ising model (2 x 1 clusters, h around 3, the held-out h = 3.0 excluded)
    predicts the stencil blocks of X, and a 12 x 12 lattice at h = 3.0 started from the prediction
    reaches the 1e-6 residual in fewer sweeps than from the cold start, at the same energy and
    with the same certificate."""
    from paper_2106_02682_gb300.warmstart import StencilWarmStart
    cluster, big = (2, 1), (12, 12)
    sw = StencilWarmStart(cluster, 2, "tfim")
    try:
        loss = sw.train((8, 8), [2.5, 2.75, 3.25, 3.5], tol=1e-6, train_steps=3000)
        assert loss < 0.05
        ham = ve.ve_ham_tfim(2, 1.0, 3.0)
        sweeps, energy, bound = {}, {}, {}
        for warm in (False, True):
            h = ve.ve_create(big, cluster, ham)
            try:
                if warm:
                    sw.apply(h, big, 3.0)
                code, st = ve.ve_iterate(h, 40000, 1e-6)
                assert code == 0
                sweeps[warm], energy[warm] = st.iter, st.energy_per_spin
                bound[warm] = ve.ve_bound(h).bound_per_spin
            finally:
                ve.ve_destroy(h)
        assert sweeps[True] < 0.9 * sweeps[False], sweeps
        assert abs(energy[True] - energy[False]) < 1e-4, energy
        assert abs(bound[True] - bound[False]) < 1e-4, bound
    finally:
        sw.close()
