"""Pins of the general (non-translation-invariant) Algorithm-5 oracle (oracle/alg5.py) against
facts fixed by the paper and the mathematics, independent of the oracle's own formulas:

  * on a periodic chain built from its spin terms, Algorithm 5 reproduces the translation-
    invariant Algorithm 6 (pinned separately) sweep by sweep;
  * with two clusters the pair marginal is the whole state, so the relaxation is exact
    (Sec. 2.3) and the certified bound converges to the exact-diagonalisation energy;
  * with no inter-cluster terms the ground state is a product state and the bound converges
    to the sum of the clusters' lowest eigenvalues;
  * the certified bound never exceeds E_0 for arbitrary multipliers and PSD X (weak duality);
  * relabelling the clusters (which turns pairs (i, j) into (j, i)) permutes the iterates and
    leaves energy, residual and bound unchanged.
"""
import numpy as np
import pytest

from oracle import alg5, models
from oracle import ve_oracle as vo
from paper_2106_02682_gb300 import synth


def _blocks(terms, L):
    bonds = [(int(s), int(t), B) for (s, t), B in zip(terms['bond_sites'], terms['bond_ops'])]
    return models.general_blocks(terms['nspins'], L, terms['onsite'], bonds), bonds


def _general(terms, L, **kw):
    blocks, bonds = _blocks(terms, L)
    pb = alg5.GeneralProblem(blocks, **kw)
    s5 = alg5.general_setup(blocks)
    return pb, s5, bonds


def test_periodic_chain_from_terms_reproduces_algorithm_6():
    n, L, J, h = 8, 2, 1.0, 0.9
    onsite, bonds = models.tfim_terms(J, h, 1)
    ti = vo.Problem(models.cluster_model((n,), (L,), onsite, bonds))
    st6 = vo.initial_state(ti)
    terms = dict(nspins=n, onsite=np.broadcast_to(onsite, (n, 2, 2)),
                 bond_sites=np.array([(s, (s + 1) % n) for s in range(n)]),
                 bond_ops=np.broadcast_to(bonds[0][1], (n, 4, 4)))
    pb, s5, _ = _general(terms, L)
    st5 = alg5.initial_state(pb, s5)
    for _ in range(6):
        d6 = vo.iterate(ti, st6)
        d5 = alg5.iterate(pb, s5, st5)
        assert d5['energy'] == pytest.approx(d6['energy'], abs=1e-13)
        assert d5['feas_err'] == pytest.approx(d6['feas_err'], rel=1e-10)
    v5 = alg5.ti_view(pb, s5, st5)
    for key in ('rho0', 'rt', 'lam', 'lam1', 'lam2', 'X'):
        np.testing.assert_allclose(v5[key], st6[key], atol=1e-12)
    b5 = alg5.certified_bound(pb, s5, st5)['bound_per_spin']
    b6 = vo.certified_bound(ti, st6)['bound_per_spin']
    assert b5 == pytest.approx(b6, abs=1e-10)


@pytest.mark.parametrize("kind,L,seed", [("tfim", 1, 11), ("xxz", 1, 11), ("xxz", 2, 4)])
def test_two_clusters_are_exact(kind, L, seed):
    terms = synth.disordered_chain(2 * L, kind, alpha=1.0, seed=seed)
    pb, s5, bonds = _general(terms, L)
    e0 = models.exact_ground_energy_terms(terms['nspins'], terms['onsite'], bonds)
    st = alg5.initial_state(pb, s5)
    alg5.run(pb, s5, st, 3000, tol=1e-11)
    b = alg5.certified_bound(pb, s5, st)
    assert b['bound_per_spin'] * terms['nspins'] <= e0 + 1e-9
    assert b['bound_per_spin'] * terms['nspins'] == pytest.approx(e0, abs=1e-8)
    assert st['energy'] * terms['nspins'] == pytest.approx(e0, abs=1e-8)


def test_two_clusters_bound_closes_in_from_below():
    # the disordered Ising pair of 2-spin clusters converges slowly; its bound stays below E_0
    # and the gap shrinks
    terms = synth.disordered_chain(4, "tfim", alpha=1.0, seed=11)
    pb, s5, bonds = _general(terms, 2)
    e0 = models.exact_ground_energy_terms(4, terms['onsite'], bonds)
    st = alg5.initial_state(pb, s5)
    gaps = []
    for _ in range(3):
        alg5.run(pb, s5, st, 500)
        gaps.append(e0 - 4 * alg5.certified_bound(pb, s5, st)['bound_per_spin'])
    assert all(g >= -1e-12 for g in gaps)
    assert gaps[0] > gaps[1] > gaps[2] and gaps[2] < 5e-4


def test_no_inter_cluster_terms_gives_the_product_ground_state():
    n, L = 6, 2
    full = synth.disordered_chain(n, "tfim", seed=5)
    keep = [(s, t) for s, t in full['bond_sites'] if s // L == t // L]
    sel = [k for k, (s, t) in enumerate(full['bond_sites']) if s // L == t // L]
    terms = dict(nspins=n, onsite=full['onsite'], bond_sites=np.array(keep),
                 bond_ops=full['bond_ops'][sel])
    pb, s5, _ = _general(terms, L)
    exact = sum(np.linalg.eigvalsh(H)[0] for H in s5['Hi'])
    st = alg5.initial_state(pb, s5)
    alg5.run(pb, s5, st, 3000, tol=1e-11)
    b = alg5.certified_bound(pb, s5, st)
    assert b['bound_per_spin'] * n <= exact + 1e-9
    assert b['bound_per_spin'] * n == pytest.approx(exact, abs=1e-6)


def test_bound_is_below_the_ground_energy_for_arbitrary_multipliers():
    n, L = 6, 1
    terms = synth.disordered_chain(n, "tfim", alpha=1.5, seed=3)
    pb, s5, bonds = _general(terms, L)
    e0 = models.exact_ground_energy_terms(n, terms['onsite'], bonds)
    rng = np.random.default_rng(7)
    K, m, D = len(s5['pairs']), pb.m, pb.D
    for draw in range(20):
        st = alg5.initial_state(pb, s5)
        st['lam1'] = rng.normal(size=(K, m, m))
        st['lam2'] = rng.normal(size=(K, m, m))
        st['lam1'] = 0.5 * (st['lam1'] + np.swapaxes(st['lam1'], 1, 2))
        st['lam2'] = 0.5 * (st['lam2'] + np.swapaxes(st['lam2'], 1, 2))
        Z = rng.normal(size=(n * D, n * D)) * 0.2
        st['X'] = Z @ Z.T
        b = alg5.certified_bound(pb, s5, st)
        assert b['x_neg_correction'] < 1e-10
        assert b['bound_per_spin'] * n <= e0 + 1e-10, draw
    # and near the optimum the bound is tight to the relaxation's accuracy
    st = alg5.initial_state(pb, s5)
    alg5.run(pb, s5, st, 600)
    b = alg5.certified_bound(pb, s5, st)
    assert e0 - 0.05 * n < b['bound_per_spin'] * n <= e0


def test_relabelling_clusters_permutes_the_iterates():
    n, L = 6, 2
    N = n // L
    terms = synth.disordered_chain(n, "xxz", alpha=1.0, seed=21)
    perm = np.array([2, 0, 1])          # cluster c -> perm[c]
    relabel = lambda s: int(perm[s // L] * L + s % L)
    t2 = dict(nspins=n, onsite=np.empty_like(terms['onsite']),
              bond_sites=np.array([(relabel(s), relabel(t)) for s, t in terms['bond_sites']]),
              bond_ops=terms['bond_ops'])
    for s in range(n):
        t2['onsite'][relabel(s)] = terms['onsite'][s]
    pa, sa, _ = _general(terms, L)
    pb, sb, _ = _general(t2, L)
    sta, stb = alg5.initial_state(pa, sa), alg5.initial_state(pb, sb)
    for _ in range(25):
        da = alg5.iterate(pa, sa, sta)
        db = alg5.iterate(pb, sb, stb)
        assert db['energy'] == pytest.approx(da['energy'], abs=1e-12)
        assert db['feas_err'] == pytest.approx(da['feas_err'], rel=1e-9, abs=1e-14)
    np.testing.assert_allclose(stb['rho'][perm], sta['rho'], atol=1e-12)
    D = pa.D
    Xa = sta['X'].reshape(N, D, N, D)
    Xb = stb['X'].reshape(N, D, N, D)[perm][:, :, perm]
    np.testing.assert_allclose(Xb, Xa, atol=1e-12)
    ba = alg5.certified_bound(pa, sa, sta)['bound_per_spin']
    bb = alg5.certified_bound(pb, sb, stb)['bound_per_spin']
    assert bb == pytest.approx(ba, abs=1e-11)


def test_state_packing_round_trips():
    terms = synth.disordered_chain(4, "tfim", seed=2)
    pb, s5, _ = _general(terms, 1)
    st = alg5.initial_state(pb, s5)
    alg5.iterate(pb, s5, st)
    v = alg5.pack_state(pb, s5, st)
    st2 = alg5.unpack_state(pb, s5, v)
    for key in ('rho', 'rt', 'lam', 'lam1', 'lam2', 'X'):
        np.testing.assert_array_equal(st2[key], st[key])
