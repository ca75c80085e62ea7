"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks an oracle function against something other than itself: a literal
definition written with Kronecker products and traces, an adjoint identity, a dense solve,
a closed form, exact diagonalisation, the un-reduced Algorithm 5, or the paper's printed
values (tests/golden/).
"""
import os

import numpy as np
import pytest

from oracle import alg5
from oracle import models as mo
from oracle import ve_oracle as vo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(20210604)


def sym(A):
    return 0.5 * (A + A.T)


def unit(m, a, b):
    E = np.zeros((m, m))
    E[a, b] = 1.0
    return E


# ------------------------------------------------------------------ partial traces / lifts

@pytest.mark.parametrize("m", [2, 4])
def test_partial_traces_on_products(m):
    A, B = rng.normal(size=(m, m)), rng.normal(size=(m, m))
    rho = np.kron(A, B)
    np.testing.assert_allclose(vo.A1(rho), A * np.trace(B), atol=1e-12)
    np.testing.assert_allclose(vo.A2(rho), np.trace(A) * B, atol=1e-12)


@pytest.mark.parametrize("m", [2, 4])
def test_partial_trace_literal_and_adjoints(m):
    rho = rng.normal(size=(m * m, m * m))
    I = np.eye(m)
    lit1 = sum(np.kron(I, I[:, [b]]).T @ rho @ np.kron(I, I[:, [b]]) for b in range(m))
    lit2 = sum(np.kron(I[:, [a]], I).T @ rho @ np.kron(I[:, [a]], I) for a in range(m))
    np.testing.assert_allclose(vo.A1(rho), lit1, atol=1e-12)
    np.testing.assert_allclose(vo.A2(rho), lit2, atol=1e-12)
    Y = rng.normal(size=(m, m))
    np.testing.assert_allclose(vo.A1_adj(Y), np.kron(Y, I), atol=0)
    np.testing.assert_allclose(vo.A2_adj(Y), np.kron(I, Y), atol=0)
    assert abs(np.sum(vo.A1(rho) * Y) - np.sum(rho * vo.A1_adj(Y))) < 1e-11
    assert abs(np.sum(vo.A2(rho) * Y) - np.sum(rho * vo.A2_adj(Y))) < 1e-11


# ------------------------------------------------------------------ the G map (Sec. 2.2)

@pytest.mark.parametrize("m", [2, 4])
def test_G_blocks_match_trace_definition(m):
    rho = rng.normal(size=(m * m, m * m))
    rho0 = rng.normal(size=(m, m))
    G = vo.G_pair(rho)
    G0 = vo.G_00(rho0)
    for a in range(m):
        for b in range(m):
            for c in range(m):
                for d in range(m):
                    Oab, Ocd = unit(m, a, b), unit(m, c, d)
                    assert abs(G[a * m + b, c * m + d] - np.trace(np.kron(Oab.T, Ocd) @ rho)) < 1e-12
                    assert abs(G0[a * m + b, c * m + d] - np.trace(Oab.T @ Ocd @ rho0)) < 1e-12


@pytest.mark.parametrize("m", [2, 4])
def test_G_adjoints_match_operator_sums(m):
    X = rng.normal(size=(m * m, m * m))
    S = np.zeros((m * m, m * m))
    S0 = np.zeros((m, m))
    for a in range(m):
        for b in range(m):
            for c in range(m):
                for d in range(m):
                    x = X[a * m + b, c * m + d]
                    S += x * np.kron(unit(m, a, b).T, unit(m, c, d))
                    S0 += x * unit(m, a, b).T @ unit(m, c, d)
    np.testing.assert_allclose(vo.G_pair_adj(X).T, S, atol=1e-12)
    np.testing.assert_allclose(vo.G_00_adj(X), S0, atol=1e-12)
    rho = rng.normal(size=(m * m, m * m))
    assert abs(np.sum(vo.G_pair(rho) * X) - np.sum(rho * vo.G_pair_adj(X))) < 1e-10


@pytest.mark.parametrize("spins_per_cluster", [1, 2])
def test_G_is_psd_on_true_marginals(spins_per_cluster):
    """The global matrix G of the marginals of any state of 3 clusters is PSD (Eq. (sdpC4))."""
    L = spins_per_cluster
    m, n = 2 ** L, 3 * L
    psi = rng.normal(size=2 ** n)
    psi /= np.linalg.norm(psi)
    T = psi.reshape([m, m, m])

    def rdm(keep):
        rest = [i for i in range(3) if i not in keep]
        t = np.transpose(T, list(keep) + rest).reshape(m ** len(keep), -1)
        return t @ t.T

    D = m * m
    G = np.zeros((3 * D, 3 * D))
    for i in range(3):
        G[i * D:(i + 1) * D, i * D:(i + 1) * D] = vo.G_00(rdm([i]))
        for j in range(i + 1, 3):
            g = vo.G_pair(rdm([i, j]))
            G[i * D:(i + 1) * D, j * D:(j + 1) * D] = g
            G[j * D:(j + 1) * D, i * D:(i + 1) * D] = g.T
    assert np.allclose(G, G.T)
    assert np.linalg.eigvalsh(G)[0] > -1e-12


@pytest.mark.parametrize("m", [2, 4])
def test_effective_hamiltonians_carry_the_lagrangian_term(m):
    """<H_0[X], rho0> = <H_0, rho0> - <X_00, G_00[rho0]> and, for symmetric rho,
    <H_0d[X], rho> = <H_0d, rho> - 2 <X, G_0d[rho]>  (Eq. (effHam) and the term -Tr[X G])."""
    D = m * m
    X00 = sym(rng.normal(size=(D, D)))
    H0 = sym(rng.normal(size=(m, m)))
    rho0 = sym(rng.normal(size=(m, m)))
    lhs = np.sum(vo.eff_ham_0(H0, X00) * rho0)
    assert abs(lhs - (np.sum(H0 * rho0) - np.sum(X00 * vo.G_00(rho0)))) < 1e-10
    X = rng.normal(size=(D, D))
    H = sym(rng.normal(size=(D, D)))
    rho = sym(rng.normal(size=(D, D)))
    Hp = vo.eff_ham_pair(H, X)
    assert np.allclose(Hp, Hp.T)
    assert abs(np.sum(Hp * rho) - (np.sum(H * rho) - 2 * np.sum(X * vo.G_pair(rho)))) < 1e-9


# ------------------------------------------------------------------ closed-form solve

@pytest.mark.parametrize("m", [2, 4])
def test_T_inverse_equals_dense_solve(m):
    mu, nu = 10.0, 10.0
    D = m * m
    I = np.eye(m)

    def T(Y):   # mu + nu A1^*A1 + nu A2^*A2 written with Kronecker products
        t2 = sum(np.kron(I, I[:, [b]]).T @ Y @ np.kron(I, I[:, [b]]) for b in range(m))
        t1 = sum(np.kron(I[:, [a]], I).T @ Y @ np.kron(I[:, [a]], I) for a in range(m))
        return mu * Y + nu * np.kron(t2, I) + nu * np.kron(I, t1)

    Tmat = np.stack([T(e.reshape(D, D)).ravel() for e in np.eye(D * D)], axis=1)
    Y = rng.normal(size=(D, D))
    dense = np.linalg.solve(Tmat, Y.ravel()).reshape(D, D)
    np.testing.assert_allclose(vo.T_inverse(Y, mu, nu), dense, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(T(vo.T_inverse(Y, mu, nu)), Y, atol=1e-12)


# ------------------------------------------------------------------ PSD projection

@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n", [2, 4, 16])
def test_projection_is_the_nearest_psd_matrix(n, complex_):
    C = rng.normal(size=(n, n)) + (1j * rng.normal(size=(n, n)) if complex_ else 0)
    C = 0.5 * (C + np.conj(C.T))
    P = vo.proj_psd(C)
    assert np.allclose(P, np.conj(P.T), atol=1e-13)
    assert np.linalg.eigvalsh(P)[0] > -1e-12                      # PSD
    assert np.linalg.eigvalsh(P - C)[0] > -1e-12                  # Moreau: P - C >= 0
    assert abs(np.vdot(P, P - C)) < 1e-11                         # <P, P - C> = 0
    np.testing.assert_allclose(vo.proj_psd(P), P, atol=1e-12)    # idempotent
    dist = np.linalg.norm(P - C)
    for _ in range(50):
        B = rng.normal(size=(n, n)) + (1j * rng.normal(size=(n, n)) if complex_ else 0)
        S = P + 0.05 * B @ np.conj(B.T)
        assert np.linalg.norm(S - C) >= dist - 1e-12


def test_projection_2x2_closed_form():
    a, b, c = 0.3, 0.9, -0.5
    C = np.array([[a, b], [b, c]])
    lam = 0.5 * (a + c) + np.sqrt(0.25 * (a - c) ** 2 + b * b)
    v = np.array([b, lam - a])
    v /= np.linalg.norm(v)
    np.testing.assert_allclose(vo.proj_psd(C), lam * np.outer(v, v), atol=1e-14)


# ------------------------------------------------------------------ block-DFT projection

def _random_first_row(M, D):
    N = int(np.prod(M))
    neg = vo.neg_index(M)
    X = rng.normal(size=(N, D, D))
    X = 0.5 * (X + np.swapaxes(X[neg], 1, 2))      # X_{0,-d} = X_{0,d}^T
    return X


def _dense_circulant(X, M):
    N, D = X.shape[0], X.shape[1]
    offs = vo.lattice_offsets(M)
    full = np.zeros((N * D, N * D))
    for i in range(N):
        for j in range(N):
            d = np.ravel_multi_index(tuple((offs[j] - offs[i]) % np.array(M)), M)
            full[i * D:(i + 1) * D, j * D:(j + 1) * D] = X[d]
    return full


@pytest.mark.parametrize("M", [(2,), (3,), (5,), (6,), (2, 3), (3, 3)])
def test_block_dft_projection_equals_dense_projection(M):
    D = 4
    X = _random_first_row(M, D)
    dense = vo.proj_psd(_dense_circulant(X, M))[:D].reshape(D, -1, D).transpose(1, 0, 2)
    via_dft = np.real(vo._lattice_dft(vo.proj_psd(vo._lattice_dft(X, M, False)), M, True))
    np.testing.assert_allclose(via_dft, dense, atol=1e-12)
    # eigen-blocks: the spectrum of the block-circulant matrix is that of the unnormalised DFT
    C = vo._lattice_dft(X, M, False) * np.sqrt(int(np.prod(M)))
    ev = np.sort(np.linalg.eigvalsh(C).ravel())
    np.testing.assert_allclose(ev, np.linalg.eigvalsh(_dense_circulant(X, M)), atol=1e-11)


def test_pair_counts():
    for N in [2, 5, 8]:
        np.testing.assert_array_equal(vo.pair_counts((N,))[1:], N - np.arange(1, N))
    for M in [(2, 3), (4, 4), (3, 5)]:
        N = int(np.prod(M))
        c = vo.pair_counts(M)
        neg = vo.neg_index(M)
        assert c[0] == 0 and c[1:].sum() == N * (N - 1) // 2
        np.testing.assert_array_equal(c[1:] + c[neg[1:]], N)


# ------------------------------------------------------------------ models

def _cluster_marginals(psi, lattice, cluster, model):
    n = int(np.prod(lattice))
    dim = len(lattice)
    sites = mo.lattice_sites(lattice)

    def members(c):
        out = [s for s in sites if tuple(s[p] // cluster[p] for p in range(dim)) == tuple(c)]
        out.sort(key=lambda s: np.ravel_multi_index(tuple(s[p] % cluster[p] for p in range(dim)),
                                                    cluster))
        return [sites.index(s) for s in out]

    T = psi.reshape([2] * n)

    def rdm(keep):
        rest = [i for i in range(n) if i not in keep]
        t = np.transpose(T, keep + rest).reshape(2 ** len(keep), -1)
        return t @ t.T

    offs = vo.lattice_offsets(model['M'])
    rho0 = rdm(members(offs[0]))
    pairs = np.array([rdm(members(offs[0]) + members(offs[d])) for d in range(1, len(offs))])
    return rho0, pairs


@pytest.mark.parametrize("lattice,cluster,kind", [
    ((6,), (1,), "tfim"), ((6,), (2,), "xxz"), ((8,), (2,), "tfim"), ((6,), (3,), "tfim"),
    ((4, 2), (1, 1), "xxz"), ((4, 4), (2, 1), "tfim"), ((4, 4), (2, 2), "xxz")])
def test_cluster_blocks_reproduce_the_ground_energy(lattice, cluster, kind):
    """N (Tr[H_0 rho_0] + 1/2 sum_d Tr[H_0d rho_0d]) on the marginals of the exact ground
    state equals E_0 (the TI pairwise form of Sec. 2.1 / 3.3)."""
    dim = len(lattice)
    on, bonds = mo.tfim_terms(1.0, 0.7, dim) if kind == "tfim" else mo.xxz_terms(1.0, 0.6, dim)
    model = mo.cluster_model(lattice, cluster, on, bonds)
    E0, psi = mo.exact_ground_energy(lattice, on, bonds, return_state=True)
    rho0, pairs = _cluster_marginals(psi, lattice, cluster, model)
    N = model['N']
    E = N * np.trace(model['H0'] @ rho0) + 0.5 * N * np.einsum('pij,pji->', model['Hpair'][1:], pairs)
    assert abs(E - E0) < 1e-9 * abs(E0)


@pytest.mark.parametrize("n", [2, 3, 4, 6, 8, 10])
@pytest.mark.parametrize("h", [0.3, 1.0, 1.7])
def test_jordan_wigner_matches_exact_diagonalisation(n, h):
    on, bonds = mo.tfim_terms(1.0, h, 1)
    assert abs(mo.tfim_chain_jw_energy(n, 1.0, h) - mo.exact_ground_energy((n,), on, bonds)) < 1e-9


# ------------------------------------------------------------------ the whole sweep

@pytest.mark.parametrize("lattice,cluster,kind", [
    ((3,), (1,), "tfim"), ((4,), (1,), "xxz"), ((8,), (2,), "tfim"), ((2, 2), (1, 1), "tfim"),
    ((4, 2), (2, 1), "xxz")])
def test_algorithm6_equals_algorithm5(lattice, cluster, kind):
    """Algorithm 6 (first block row, block-DFT projection) reproduces the iterates of the
    un-reduced Algorithm 5 (all pairs, dense X projection) on the same periodic lattice."""
    dim = len(lattice)
    on, bonds = mo.tfim_terms(1.0, 0.8, dim) if kind == "tfim" else mo.xxz_terms(1.0, 0.5, dim)
    pb = vo.Problem(mo.cluster_model(lattice, cluster, on, bonds))
    st6 = vo.initial_state(pb)
    s5 = alg5.setup(pb)
    st5 = alg5.initial_state(pb, s5)
    for it in range(25):
        vo.iterate(pb, st6)
        alg5.iterate(pb, s5, st5)
    v5 = alg5.ti_view(pb, s5, st5)
    for key in ['rho0', 'rt', 'lam', 'lam1', 'lam2', 'X']:
        np.testing.assert_allclose(st6[key], v5[key], atol=1e-10, err_msg=key)


@pytest.mark.parametrize("lattice,cluster,kind", [((4, 6), (2, 1), "tfim"), ((10,), (2,), "xxz"),
                                                  ((9,), (3,), "tfim")])
def test_swap_symmetry_is_preserved(lattice, cluster, kind):
    """The offsets d and -d see the same pairs of clusters from either end: H_{-d} = P H_d P,
    and from the initial state the iteration keeps rho~_{-d} = P rho~_d P, Lambda_{-d} =
    P Lambda_d P, Lambda1_{-d} = Lambda2_d, X_{-d} = X_d^T (P swaps the clusters)."""
    dim = len(lattice)
    on, bonds = mo.tfim_terms(1.0, 1.1, dim) if kind == "tfim" else mo.xxz_terms(1.0, 0.6, dim)
    pb = vo.Problem(mo.cluster_model(lattice, cluster, on, bonds))
    st = vo.initial_state(pb)
    for _ in range(60):
        vo.iterate(pb, st)
    m, D = pb.m, pb.D
    neg = vo.neg_index(pb.M)
    swap = np.eye(D)[[b * m + a for a in range(m) for b in range(m)]]
    np.testing.assert_array_equal(pb.Hpair[neg[1:] - 1], swap @ pb.Hpair @ swap)
    np.testing.assert_allclose(st['rt'][neg[1:] - 1], swap @ st['rt'] @ swap, atol=1e-12)
    np.testing.assert_allclose(st['lam'][neg[1:] - 1], swap @ st['lam'] @ swap, atol=1e-11)
    np.testing.assert_allclose(st['lam1'][neg[1:] - 1], st['lam2'], atol=1e-12)
    np.testing.assert_allclose(st['X'][neg], np.swapaxes(st['X'], 1, 2), atol=1e-12)


@pytest.mark.parametrize("lattice,cluster,kind,h", [
    ((8,), (1,), "tfim", 0.5), ((8,), (2,), "tfim", 1.0), ((10,), (2,), "tfim", 1.5),
    ((8,), (2,), "xxz", 1.0), ((4, 4), (1, 1), "tfim", 2.0), ((4, 4), (2, 1), "xxz", 0.5)])
def test_bound_is_below_exact_energy(lattice, cluster, kind, h):
    dim = len(lattice)
    on, bonds = mo.tfim_terms(1.0, h, dim) if kind == "tfim" else mo.xxz_terms(1.0, h, dim)
    pb = vo.Problem(mo.cluster_model(lattice, cluster, on, bonds))
    st = vo.initial_state(pb)
    n = int(np.prod(lattice))
    E0 = mo.exact_ground_energy(lattice, on, bonds) / n
    for it in range(400):
        vo.iterate(pb, st)
        if it % 100 == 0:
            assert vo.certified_bound(pb, st)['bound_per_spin'] <= E0 + 1e-12
    assert vo.certified_bound(pb, st)['bound_per_spin'] <= E0 + 1e-12


def test_duality_gap_closes_and_bound_tightens_with_cluster_size():
    on, bonds = mo.xxz_terms(1.0, 1.0, 1)
    out = {}
    for L in (1, 2):
        pb = vo.Problem(mo.cluster_model((8,), (L,), on, bonds))
        st = vo.initial_state(pb)
        vo.run(pb, st, 3000)
        out[L] = vo.certified_bound(pb, st)
    # 2-site clusters converge here; the certificate meets the primal energy
    assert abs(out[2]['bound_per_spin'] - out[2]['primal_per_spin']) < 1e-6
    assert out[2]['bound_per_spin'] > out[1]['bound_per_spin'] + 0.1


@pytest.mark.parametrize("lattice,cluster,exact", [((12,), (1,), -1.0), ((10,), (2,), -1.0),
                                                   ((4, 4), (1, 1), -2.0)])
def test_relaxation_is_exact_at_zero_field(lattice, cluster, exact):
    """At h = 0 the TFI relaxation is exact (Sec. 4, caption of the TFI benchmark figure)."""
    on, bonds = mo.tfim_terms(1.0, 0.0, len(lattice))
    pb = vo.Problem(mo.cluster_model(lattice, cluster, on, bonds))
    st = vo.initial_state(pb)
    vo.run(pb, st, 1500)
    cert = vo.certified_bound(pb, st)
    assert cert['bound_per_spin'] <= exact + 1e-12
    assert cert['bound_per_spin'] > exact - 1e-6
    assert abs(st['energy'] - exact) < 1e-6


def _golden():
    rows = []
    with open(os.path.join(GOLDEN, "tfi_relaxation_energies.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, c, h, e = line.split()
                rows.append((int(n), int(c), float(h), float(e)))
    return rows


@pytest.mark.parametrize("h", [0.5, 1.0, 1.5])
def test_paper_table_single_site_clusters(h):
    """TFI 100x1 with 1x1 clusters (4-decimal table): after the paper's 10 000 iterations the
    relaxation energy per site matches, and the certified bound lies below it."""
    ref = [e for n, c, hh, e in _golden() if n == 100 and c == 1 and hh == h][0]
    on, bonds = mo.tfim_terms(1.0, h, 1)
    pb = vo.Problem(mo.cluster_model((100,), (1,), on, bonds))
    st = vo.initial_state(pb)
    vo.run(pb, st, 10000)
    assert abs(st['energy'] - ref) <= 1.5e-4
    assert vo.certified_bound(pb, st)['bound_per_spin'] <= ref + 5e-5


@pytest.mark.slow
def test_paper_table_two_site_clusters_h1():
    """TFI 20x1 with 2x1 clusters, h = 1 (6-decimal table): energy within 5e-6 after 10 000
    iterations; the certified bound lies below the printed optimum and within 5e-6 of it."""
    ref = [e for n, c, hh, e in _golden() if n == 20 and c == 2 and hh == 1.0][0]
    on, bonds = mo.tfim_terms(1.0, 1.0, 1)
    pb = vo.Problem(mo.cluster_model((20,), (2,), on, bonds))
    st = vo.initial_state(pb)
    vo.run(pb, st, 10000)
    cert = vo.certified_bound(pb, st)
    assert abs(st['energy'] - ref) < 5e-6
    assert ref - 5e-6 < cert['bound_per_spin'] <= ref + 1e-7
    assert cert['bound_per_spin'] <= mo.tfim_chain_jw_energy(20, 1.0, 1.0) / 20


def test_bound_below_jordan_wigner_energy_long_chain():
    on, bonds = mo.tfim_terms(1.0, 1.0, 1)
    pb = vo.Problem(mo.cluster_model((64,), (2,), on, bonds))
    st = vo.initial_state(pb)
    vo.run(pb, st, 300)
    assert vo.certified_bound(pb, st)['bound_per_spin'] <= mo.tfim_chain_jw_energy(64, 1.0, 1.0) / 64


# ------------------------------------------------------------------ warm-start network (CPU reference)

def test_mlp_reference_gradient_matches_finite_differences():
    from oracle import mlp
    shapes = mlp.layer_shapes(2, 7, 2, 3)
    n = sum(o * i + o for o, i in shapes)
    params = rng.normal(scale=0.5, size=n)
    x = rng.normal(size=(5, 2))
    t = rng.normal(size=(5, 3))
    loss, g = mlp.loss_grad(params, shapes, x, t)
    fd = np.empty(n)
    h = 1e-6
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (mlp.loss_grad(params + e, shapes, x, t)[0] - mlp.loss_grad(params - e, shapes, x, t)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)
    # the loss is the stated mean of squared residuals / 2
    y = mlp.forward(params, shapes, x)[-1]
    assert abs(loss - 0.5 * np.mean((y - t) ** 2)) < 1e-15
