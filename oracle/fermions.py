"""Spinless fermions for the oracle: the models of the paper's fermionic section (Eq.
(spinlessFerm) and its long-range form Eq. (spinlessFermLR)) on a periodic ring, their cluster
blocks under a Jordan-Wigner transformation (JWT) chosen per cluster and per pair of clusters
(Eq. (sdpFerm)), exact diagonalisation in Fock space, and the free-fermion energy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Conventions, as in the paper's JWT: a site's basis is (empty, occupied); a_i^dagger acts as
sigma^z on every site before i in the chosen ordering, as [[0, 0], [1, 0]] on site i, and as the
identity after it.  Clusters are runs of L consecutive sites; a cluster's own ordering is its
sites in increasing order, and a pair (gamma < delta) orders gamma's sites before delta's, so a
cluster basis index has the cluster's first site as its most significant bit, as for spins.
"""
import numpy as np

SM = np.array([[0.0, 0.0], [1.0, 0.0]])   # creation on one site
SZ = np.diag([1.0, -1.0])
N1 = np.diag([0.0, 1.0])                  # number operator on one site


def creation_ops(nsites):
    """a_i^dagger for i = 0 .. nsites-1 as dense 2^nsites matrices (JWT in this order)."""
    ops = []
    for i in range(nsites):
        factors = [SZ] * i + [SM] + [np.eye(2)] * (nsites - i - 1)
        op = np.array([[1.0]])
        for f in factors:
            op = np.kron(op, f)
        ops.append(op)
    return ops


def ring_terms(M, U, long_range=False):
    """Terms of Eq. (spinlessFerm) on a periodic ring of M sites (i ~ j: ring neighbours, each
    bond once), or of Eq. (spinlessFermLR): the same hopping plus U sum_{i != j} (n_i - 1/2)
    (n_j - 1/2) / d(i, j), d the distance on the ring (every unordered pair carries 2 U / d).
    Returns (hops [(i, j, t)] meaning t (a_i^dagger a_j + a_j^dagger a_i), pairs [(i, j, v)]
    meaning v (n_i - 1/2)(n_j - 1/2))."""
    bonds = sorted({tuple(sorted((i, (i + 1) % M))) for i in range(M)})
    hops = [(i, j, -1.0) for i, j in bonds]
    if not long_range:
        pairs = [(i, j, float(U)) for i, j in bonds]
    else:
        pairs = []
        for i in range(M):
            for j in range(i + 1, M):
                d = min(j - i, M - (j - i))
                pairs.append((i, j, 2.0 * U / d))
    return hops, pairs


def _term_matrix(adag, pos, hop=None, pair=None):
    dim = adag[0].shape[0]
    eye = np.eye(dim)
    if hop is not None:
        i, j, t = hop
        ai, aj = adag[pos[i]], adag[pos[j]]
        return t * (ai @ aj.T + aj @ ai.T)
    i, j, v = pair
    ni, nj = adag[pos[i]] @ adag[pos[i]].T, adag[pos[j]] @ adag[pos[j]].T
    return v * (ni - 0.5 * eye) @ (nj - 0.5 * eye)


def full_hamiltonian(M, U, long_range=False):
    """The whole-ring Hamiltonian in Fock space (JWT in site order), dense; M <= 12."""
    adag = creation_ops(M)
    pos = list(range(M))
    hops, pairs = ring_terms(M, U, long_range)
    H = np.zeros((2 ** M, 2 ** M))
    for h in hops:
        H += _term_matrix(adag, pos, hop=h)
    for p in pairs:
        H += _term_matrix(adag, pos, pair=p)
    return H


def exact_ground_energy(M, U, long_range=False):
    return float(np.linalg.eigvalsh(full_hamiltonian(M, U, long_range))[0])


def free_fermion_energy(M):
    """E_0 at U = 0 with no particle-number constraint: the sum of the negative eigenvalues of
    the ring's hopping matrix, -2 cos(2 pi k / M)."""
    eps = -2.0 * np.cos(2.0 * np.pi * np.arange(M) / M)
    return float(np.sum(eps[eps < 0]))


def fermion_blocks(M, L, U, long_range=False):
    """Cluster blocks of Eq. (sdpFerm): H_gamma = J_gamma(sum of the terms inside cluster gamma),
    H_gamma,delta = J_gamma,delta(sum of the terms between the two clusters), the JWTs ordered as
    in the module docstring.  Same layout as models.general_blocks (pairs gamma < delta in
    lexicographic order)."""
    assert M % L == 0 and M // L >= 2
    N = M // L
    m = 2 ** L
    D = m * m
    hops, pairs = ring_terms(M, U, long_range)
    terms = [("hop", t) for t in hops] + [("pair", t) for t in pairs]
    cl = lambda s: s // L
    a1 = creation_ops(L)
    a2 = creation_ops(2 * L)
    Hi = np.zeros((N, m, m))
    cl_pairs = [(g, d) for g in range(N) for d in range(g + 1, N)]
    index = {gd: p for p, gd in enumerate(cl_pairs)}
    Hij = np.zeros((len(cl_pairs), D, D))
    for kind, t in terms:
        i, j = t[0], t[1]
        ci, cj = cl(i), cl(j)
        if ci == cj:
            pos = {i: i % L, j: j % L}
            Hi[ci] += _term_matrix(a1, pos, **{kind: t})
        else:
            g, d = min(ci, cj), max(ci, cj)
            pos = {s: (s % L if cl(s) == g else L + s % L) for s in (i, j)}
            Hij[index[(g, d)]] += _term_matrix(a2, pos, **{kind: t})
    return dict(Hi=Hi, Hij=Hij, pairs=cl_pairs, N=N, L=L, m=m, D=D)


def parity_signs(m):
    """The sign pattern of the fermionic global matrix's off-diagonal blocks (Eq. (sdpFerm)
    with the complete collection of matrix units E_ab of each cluster): in the pair's JWT an
    operator E_cd of the second cluster that changes the fermion parity (p(c) != p(d), p the
    parity of the occupation bits) carries the parity string P of the first cluster, and
    (E_ab^dagger P) = (-1)^p(a) E_ba.  Entry (a, b), (c, d) of the D x D mask is
    (-1)^(p(a) (p(c) + p(d)))."""
    p = np.array([bin(x).count("1") & 1 for x in range(m)])
    a = p[:, None, None, None]
    cd = (p[None, None, :, None] + p[None, None, None, :]) % 2
    sign = np.where((a * cd) % 2 == 1, -1.0, 1.0)
    return np.broadcast_to(sign, (m, m, m, m)).reshape(m * m, m * m).copy()
