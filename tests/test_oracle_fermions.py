"""Pins of the fermionic relaxation in the oracle (oracle/fermions.py, oracle/alg5.py with
fermionic=True): the spinless-fermion models of the paper's fermionic section with a
Jordan-Wigner transformation per cluster and per pair of clusters (Eq. (sdpFerm)).

  * with two clusters the pair's JWT is a global one, so the cluster blocks reproduce the
    Fock-space spectrum of the whole ring;
  * at U = 0 the relaxation is exact (the paper, citing Lin & Lindsey): the converged energy is
    the free-fermion ground energy, the sum of the ring's negative hopping eigenvalues;
  * the parity signs matter: with the spin global matrix the same blocks relax strictly below;
  * interacting rings (short- and long-range): the certified bound stays below the Fock-space
    E_0 and meets the primal energy as the iteration converges.
"""
import numpy as np
import pytest

from oracle import alg5
from oracle import fermions as fm


def _solve(M, L, U, sweeps, fermionic=True, long_range=False):
    blocks = fm.fermion_blocks(M, L, U, long_range=long_range)
    pb = alg5.GeneralProblem(blocks, fermionic=fermionic)
    s5 = alg5.general_setup(blocks)
    st = alg5.initial_state(pb, s5)
    diag = alg5.run(pb, s5, st, sweeps)
    return pb, s5, st, diag


def test_free_fermion_energy_closed_form_matches_fock_space():
    for M in (4, 6, 8, 10):
        assert fm.free_fermion_energy(M) == pytest.approx(fm.exact_ground_energy(M, 0.0), abs=1e-12)


@pytest.mark.parametrize("L,U,lr", [(1, 1.5, False), (2, 2.0, False), (2, 1.0, True), (3, 0.7, False)])
def test_two_cluster_blocks_reproduce_the_fock_space_spectrum(L, U, lr):
    M = 2 * L
    b = fm.fermion_blocks(M, L, U, long_range=lr)
    m = b['m']
    H = np.kron(b['Hi'][0], np.eye(m)) + np.kron(np.eye(m), b['Hi'][1]) + b['Hij'][0]
    np.testing.assert_allclose(np.linalg.eigvalsh(H),
                               np.linalg.eigvalsh(fm.full_hamiltonian(M, U, lr)), atol=1e-12)


def test_parity_sign_mask():
    s = fm.parity_signs(2)
    # single site: the only sign flips are a = occupied with an odd (c, d)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                for d in range(2):
                    want = -1.0 if (a == 1 and c != d) else 1.0
                    assert s[a * 2 + b, c * 2 + d] == want
    s4 = fm.parity_signs(4)
    assert s4.shape == (16, 16) and set(np.unique(s4)) == {-1.0, 1.0}


# 2-site clusters; with single-site clusters the iteration at mu = nu = 10, eps = 2 oscillates
# (energy swinging by ~1 after thousands of sweeps), as the paper's parameters do on the
# Heisenberg model with 1 x 1 clusters
@pytest.mark.parametrize("M,L", [(10, 2), (12, 2)])
def test_relaxation_is_exact_for_free_fermions(M, L):
    _, _, st, diag = _solve(M, L, 0.0, 2400)
    assert diag['residual'] < 1e-9
    assert st['energy'] * M == pytest.approx(fm.free_fermion_energy(M), abs=1e-8)


def test_spin_global_matrix_relaxes_below_the_fermionic_one():
    M, L = 8, 2
    _, _, sf, _ = _solve(M, L, 0.0, 1500)
    _, _, ss, _ = _solve(M, L, 0.0, 1500, fermionic=False)
    e0 = fm.free_fermion_energy(M)
    assert sf['energy'] * M == pytest.approx(e0, abs=1e-7)
    assert ss['energy'] * M < e0 - 0.1


@pytest.mark.parametrize("U,lr", [(2.0, False), (1.0, True)])
def test_interacting_bound_is_below_exact_and_meets_the_primal(U, lr):
    M, L = 8, 2
    pb, s5, st, diag = _solve(M, L, U, 2500, long_range=lr)
    e0 = fm.exact_ground_energy(M, U, lr)
    b = alg5.certified_bound(pb, s5, st)
    assert b['bound_per_spin'] * M <= e0 + 1e-10
    assert st['energy'] * M <= e0 + 1e-6
    assert abs(b['bound_per_spin'] - st['energy']) * M < 1e-4
