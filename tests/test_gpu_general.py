"""GPU parity of the general (non-translation-invariant) solver -- Algorithm 5 -- and of its
whole-GPU dense PSD projection, through the C ABI against the CPU oracle (oracle/alg5.py,
numpy eigh), on the same seeded inputs.

Tolerances: float64 results are held to 1e-10 relative to the largest entry of the compared
array, scaled by max(1, n / 64) for an n x n eigensolve (the Jacobi and LAPACK backward errors
both grow like n eps ||A||; the X step of a 128-spin chain is 512 x 512).  Scalars (energy,
residual, bound) use the same scale.
"""
import numpy as np
import pytest

import __graft_entry__
from oracle import alg5, models
from oracle.ve_oracle import proj_psd
from paper_2106_02682_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL64 = 1e-10


def tol(n):
    return RTOL64 * max(1.0, n / 64.0)


@pytest.fixture(scope="module")
def ve():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    __graft_entry__.build()
    from paper_2106_02682_gb300 import ve as mod
    return mod


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


# ------------------------------------------------------------------ dense projection
def _dense(ve, Y, ws=None, warm=0, alias=False, first_order=False):
    n = Y.shape[0]
    nb = ve.ve_project_psd_dense_workspace_size(n)
    if ws is None:
        ws = torch.empty(nb // 8 + 32, dtype=torch.float64, device="cuda")
    yin = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    out = yin if alias else torch.empty_like(yin)
    sweeps = ve.ve_project_psd_dense(yin.data_ptr(), out.data_ptr(), n, ws.data_ptr(), nb, warm,
                                     first_order=first_order)
    return out.cpu().numpy(), sweeps, ws


@pytest.mark.parametrize("n", [2, 6, 24, 64, 130, 256, 512, 1024])
def test_dense_projection_matches_the_oracle(ve, n):
    Ys = synth.symmetric_batch(2, n, seed=n)  # matrix 0 has repeated eigenvalues +1 / -1 / 0
    for Y in Ys:
        X, sweeps, _ = _dense(ve, Y)
        ref = proj_psd(Y)
        assert relerr(X, ref) < tol(n), (n, relerr(X, ref))
        assert 1 <= sweeps <= 24


@pytest.mark.parametrize("n", [64, 512])
def test_dense_projection_is_reproducible(ve, n):
    # fixed-order reductions throughout: the same input gives the same bits
    Y = synth.symmetric_batch(2, n, seed=7 + n)[1]
    Xa, sa, _ = _dense(ve, Y)
    Xb, sb, _ = _dense(ve, Y)
    assert sa == sb
    np.testing.assert_array_equal(Xa, Xb)


def test_dense_projection_warm_restart_and_aliasing(ve):
    n = 256
    rng = np.random.default_rng(3)
    Y = synth.symmetric_batch(2, n, seed=1)[1]
    X0, s0, ws = _dense(ve, Y)
    # the same matrix again from the eigenvectors just computed: one sweep confirms them
    X1, s1, ws = _dense(ve, Y, ws=ws, warm=1)
    assert s1 == 1 and s0 > 2
    assert relerr(X1, X0) < tol(n)
    # a nearby matrix from the old eigenvectors, written over its input
    E = rng.normal(size=(n, n)) * 1e-3
    Y2 = Y + 0.5 * (E + E.T)
    X2, s2, _ = _dense(ve, Y2, ws=ws, warm=1, alias=True)
    assert relerr(X2, proj_psd(Y2)) < tol(n)
    assert s2 < s0


@pytest.mark.parametrize("n", [64, 256, 512])
def test_dense_first_order_stop_is_as_accurate_as_the_sweeps(ve, n):
    # from the eigenvectors of Y, a nearby matrix: the explicit check on A = V^T Y' V ends the
    # sweeps early, with the Daleckii-Krein reconstruction when the spectrum keeps away from 0
    rng = np.random.default_rng(n)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = rng.uniform(0.05, 1.0, size=n) * rng.choice([-1.0, 1.0], size=n)
    Y = (Q * lam) @ Q.T
    _, _, ws = _dense(ve, Y)
    saved = ws.clone()
    E = rng.normal(size=(n, n)) * 1e-4
    Y2 = Y + 0.5 * (E + E.T)
    ref = proj_psd(Y2)
    Xe, se, _ = _dense(ve, Y2, ws=ws, warm=1)
    Xd, sd, _ = _dense(ve, Y2, ws=saved, warm=1, first_order=True)
    assert relerr(Xe, ref) < tol(n)
    assert relerr(Xd, ref) < tol(n)
    assert sd % 1000 < se                 # the explicit check saved sweeps
    if n == 256:
        assert sd >= 1000                  # ... and here ended with the first-order reconstruction


def test_dense_projection_of_psd_and_nsd_matrices(ve):
    n = 96
    Q, _ = np.linalg.qr(np.random.default_rng(5).normal(size=(n, n)))
    lam = np.linspace(0.1, 2.0, n)
    P = (Q * lam) @ Q.T
    X, _, _ = _dense(ve, P)
    assert relerr(X, P) < tol(n)          # PSD: unchanged
    X, _, _ = _dense(ve, -P)
    assert np.max(np.abs(X)) < tol(n)     # negative definite: zero


# ------------------------------------------------------------------ general solver
def _oracle(terms, L):
    bonds = [(int(s), int(t), B) for (s, t), B in zip(terms['bond_sites'], terms['bond_ops'])]
    blocks = models.general_blocks(terms['nspins'], L, terms['onsite'], bonds)
    pb = alg5.GeneralProblem(blocks)
    s5 = alg5.general_setup(blocks)
    return pb, s5, alg5.initial_state(pb, s5), bonds


CASES = [
    # (nspins, cluster spins, model, sweeps): X of N D = 24 ... 512
    (6, 1, "tfim", 12),
    (8, 2, "xxz", 10),
    (9, 3, "tfim", 6),     # D = 64, three clusters
    (40, 1, "tfim", 6),    # n = 160: ragged against 32-wide tiles
    (32, 2, "xxz", 5),     # n = 256, 120 pairs
]


@pytest.mark.parametrize("nspins,L,kind,sweeps", CASES)
def test_general_sweeps_match_the_oracle(ve, nspins, L, kind, sweeps):
    terms = synth.disordered_chain(nspins, kind, alpha=1.5, seed=nspins)
    pb, s5, st, _ = _oracle(terms, L)
    h = ve.ve_general_create(terms, L)
    try:
        N, m, D, K = ve.ve_general_dims(h)
        assert (N, m, D, K) == (pb.N, pb.m, pb.D, len(s5['pairs']))
        np.testing.assert_array_equal(ve.ve_general_get_state(h), alg5.pack_state(pb, s5, st))
        n = N * D
        for k in range(sweeps):
            diag = alg5.iterate(pb, s5, st)
            code, gs = ve.ve_general_iterate(h, 1)
            assert code == ve.VE_OK and gs.iter == k + 1
            assert gs.energy_per_spin == pytest.approx(diag['energy'], abs=tol(n))
            assert gs.feas_err == pytest.approx(diag['feas_err'], rel=tol(n), abs=1e-14)
        state = ve.ve_general_get_state(h)
        ref = alg5.pack_state(pb, s5, st)
        assert relerr(state, ref) < tol(n), relerr(state, ref)
        c = ve.ve_general_bound(h)
        oc = alg5.certified_bound(pb, s5, st)
        assert c.bound_per_spin == pytest.approx(oc['bound_per_spin'], abs=tol(n))
        assert c.raw_bound == pytest.approx(oc['raw_bound'], abs=tol(n) * nspins)
        assert c.x_neg_correction <= 1e-10 * nspins
    finally:
        ve.ve_general_destroy(h)


def test_general_runs_are_reproducible_and_resume_from_the_state(ve):
    terms = synth.disordered_chain(24, "tfim", alpha=2.0, seed=4)
    a = ve.ve_general_create(terms, 2)
    b = ve.ve_general_create(terms, 2)
    try:
        ve.ve_general_iterate(a, 9)
        ve.ve_general_iterate(b, 9)
        sa, sb = ve.ve_general_get_state(a), ve.ve_general_get_state(b)
        np.testing.assert_array_equal(sa, sb)
        # read, continue, set back, continue again: bit for bit on the same handle
        ve.ve_general_iterate(a, 3)
        after = ve.ve_general_get_state(a)
        ve.ve_general_set_state(b, sb)
        ve.ve_general_iterate(b, 3)
        np.testing.assert_array_equal(ve.ve_general_get_state(b), after)
    finally:
        ve.ve_general_destroy(a)
        ve.ve_general_destroy(b)


def test_general_two_clusters_reach_the_exact_ground_energy(ve):
    terms = synth.disordered_chain(4, "xxz", alpha=1.0, seed=4)
    _, _, _, bonds = _oracle(terms, 2)
    e0 = models.exact_ground_energy_terms(4, terms['onsite'], bonds)
    h = ve.ve_general_create(terms, 2)
    try:
        code, st = ve.ve_general_iterate(h, 3000, 1e-11)
        assert code == ve.VE_OK
        c = ve.ve_general_bound(h)
        assert 4 * c.bound_per_spin <= e0 + 1e-9
        assert 4 * c.bound_per_spin == pytest.approx(e0, abs=1e-8)
    finally:
        ve.ve_general_destroy(h)


def test_general_full_size_workload_matches_the_oracle(ve):
    # the benchmark instance: 128 spins, single-spin clusters, all-to-all 1/r^2 couplings
    # (8128 pairs, 512 x 512 X), three sweeps compared entry by entry
    terms = synth.disordered_chain(128, "tfim", alpha=2.0, seed=None)
    pb, s5, st, _ = _oracle(terms, 1)
    h = ve.ve_general_create(terms, 1)
    try:
        for _ in range(3):
            diag = alg5.iterate(pb, s5, st)
        code, gs = ve.ve_general_iterate(h, 3)
        n = pb.N * pb.D
        assert gs.energy_per_spin == pytest.approx(diag['energy'], abs=tol(n))
        assert relerr(ve.ve_general_get_state(h), alg5.pack_state(pb, s5, st)) < tol(n)
        c = ve.ve_general_bound(h)
        assert c.bound_per_spin == pytest.approx(alg5.certified_bound(pb, s5, st)['bound_per_spin'],
                                                 abs=tol(n))
    finally:
        ve.ve_general_destroy(h)


# ------------------------------------------------------------------ spinless fermions
FERMION_CASES = [
    # (sites, sites per cluster, U, long range, sweeps)
    (8, 2, 2.0, False, 10),
    (12, 2, 1.0, True, 6),
    (9, 3, 0.7, True, 4),
]


@pytest.mark.parametrize("M,L,U,lr,sweeps", FERMION_CASES)
def test_fermion_sweeps_match_the_oracle(ve, M, L, U, lr, sweeps):
    from oracle import fermions
    blocks = fermions.fermion_blocks(M, L, U, long_range=lr)
    pb = alg5.GeneralProblem(blocks, fermionic=True)
    s5 = alg5.general_setup(blocks)
    st = alg5.initial_state(pb, s5)
    h = ve.ve_general_create_fermions(synth.fermion_ring(M, U, long_range=lr), L)
    try:
        n = pb.N * pb.D
        for k in range(sweeps):
            diag = alg5.iterate(pb, s5, st)
            code, gs = ve.ve_general_iterate(h, 1)
            assert gs.energy_per_spin == pytest.approx(diag['energy'], abs=tol(n))
            assert gs.feas_err == pytest.approx(diag['feas_err'], rel=tol(n), abs=1e-14)
        assert relerr(ve.ve_general_get_state(h), alg5.pack_state(pb, s5, st)) < tol(n)
        c = ve.ve_general_bound(h)
        assert c.bound_per_spin == pytest.approx(alg5.certified_bound(pb, s5, st)['bound_per_spin'],
                                                 abs=tol(n))
    finally:
        ve.ve_general_destroy(h)


def test_fermion_relaxation_is_exact_at_zero_interaction_on_the_gpu(ve):
    from oracle import fermions
    M = 12
    h = ve.ve_general_create_fermions(synth.fermion_ring(M, 0.0), 2)
    try:
        code, st = ve.ve_general_iterate(h, 4000, 1e-11)
        assert code == ve.VE_OK
        assert M * st.energy_per_spin == pytest.approx(fermions.free_fermion_energy(M), abs=1e-8)
        assert M * ve.ve_general_bound(h).bound_per_spin <= fermions.free_fermion_energy(M) + 1e-9
    finally:
        ve.ve_general_destroy(h)
