"""Spin-1/2 lattice models for the oracle: site terms, cluster blocks H_0 / H_{0,delta},
full-lattice Hamiltonians for exact diagonalisation, and the Jordan-Wigner energy.

TEST INFRASTRUCTURE ONLY.  This module belongs to the CPU oracle; only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline / reference legs may import it.
The GPU solver builds its own cluster blocks in its own host code and never uses this.

Conventions (the paper fixes the physics, these fix the bookkeeping):
  * Spin basis: |0> = sigma^z eigenvalue +1, |1> = -1; an operator on k spins is a
    2^k x 2^k matrix in Kronecker order, spin 0 being the FIRST (most significant) factor.
  * A lattice is a tuple of spin extents per axis, periodic in every axis; a cluster is a
    rectangular block of spins of shape `cluster` (Sec. 2.3 "Cluster relaxation"), and
    clusters tile the lattice.  In-cluster spins are numbered row-major.
  * A pair operator on (cluster 0) x (cluster delta) has cluster 0 as the first factor,
    so its basis index is a*m + b with a the cluster-0 state and b the cluster-delta state.
  * delta is a vector of cluster offsets; its linear index is row-major over the cluster
    lattice (clusters per axis M_p = lattice_p / cluster_p).
"""
import itertools

import numpy as np

SX = np.array([[0.0, 1.0], [1.0, 0.0]])
SZ = np.array([[1.0, 0.0], [0.0, -1.0]])
# sigma^y (x) sigma^y is real although sigma^y is not.
SYSY = np.real(np.kron(np.array([[0, -1j], [1j, 0]]), np.array([[0, -1j], [1j, 0]])))


def tfim_terms(J, h, dim):
    """Transverse-field Ising site terms, Eq. (TFI): H = -h sum_i s^x_i - J sum_{i~j} s^z_i s^z_j.

    Returns (onsite 2x2, [(bond offset vector, bond 4x4)]) with one bond per lattice axis.
    """
    onsite = -h * SX
    bond = -J * np.kron(SZ, SZ)
    return onsite, [(tuple(int(a == p) for a in range(dim)), bond) for p in range(dim)]


def xxz_terms(J, Delta, dim):
    """XXZ site terms: J sum_{i~j} [s^x s^x + s^y s^y + Delta s^z s^z].

    Delta = 1, J = 1 is the antiferromagnetic Heisenberg model, Eq. (AFH).  The paper has no
    XXZ model; this anisotropic generalisation is the natural one-parameter extension.
    """
    onsite = np.zeros((2, 2))
    bond = J * (np.kron(SX, SX) + SYSY + Delta * np.kron(SZ, SZ))
    return onsite, [(tuple(int(a == p) for a in range(dim)), bond) for p in range(dim)]


def embed(op, positions, nspins):
    """Embed a k-spin operator `op` acting on spins `positions` (in op's factor order)
    into the 2^nspins dimensional space of `nspins` spins, by explicit basis enumeration."""
    k = len(positions)
    dim = 2 ** nspins
    out = np.zeros((dim, dim))
    for col in range(dim):
        bits = [(col >> (nspins - 1 - s)) & 1 for s in range(nspins)]
        sub_col = 0
        for p in positions:
            sub_col = 2 * sub_col + bits[p]
        for sub_row in range(2 ** k):
            amp = op[sub_row, sub_col]
            if amp == 0.0:
                continue
            nb = list(bits)
            for q, p in enumerate(positions):
                nb[p] = (sub_row >> (k - 1 - q)) & 1
            row = 0
            for b in nb:
                row = 2 * row + b
            out[row, col] += amp
    return out


def lattice_sites(lattice):
    return list(itertools.product(*[range(n) for n in lattice]))


def cluster_model(lattice, cluster, onsite, bonds):
    """Cluster Hamiltonian blocks for a translation-invariant lattice (Sec. 3.3).

    Every term of the full Hamiltonian is assigned to the cluster(s) it touches: a term
    inside one cluster goes to that cluster's H_i; a term coupling clusters i and j goes to
    H_ij (Sec. 2.1 pairwise form, Sec. 2.3 cluster relaxation).  By translation invariance
    only cluster 0's blocks are kept: H_0 (m x m) and H_{0,delta} (D x D, cluster 0 first)
    for each cluster offset delta, which collects EVERY term between cluster 0 and cluster
    delta, whichever end the term starts from.

    Returns dict with H0 (m,m), Hpair (N,D,D) indexed by delta's linear index (entry 0 is
    unused and zero), plus the shape bookkeeping.
    """
    lattice = tuple(lattice)
    cluster = tuple(cluster)
    dim = len(lattice)
    M = tuple(n // c for n, c in zip(lattice, cluster))
    assert all(n % c == 0 for n, c in zip(lattice, cluster))
    N = int(np.prod(M))
    L = int(np.prod(cluster))
    m = 2 ** L
    D = m * m

    def cl(s):
        return tuple(s[p] // cluster[p] for p in range(dim))

    def local(s):
        u = 0
        for p in range(dim):
            u = u * cluster[p] + s[p] % cluster[p]
        return u

    def lin(c):
        u = 0
        for p in range(dim):
            u = u * M[p] + c[p]
        return u

    zero = tuple([0] * dim)
    H0 = np.zeros((m, m))
    Hpair = np.zeros((N, D, D))
    for s in lattice_sites(lattice):
        cs = cl(s)
        if cs == zero:
            H0 += embed(onsite, [local(s)], L)
        for e, B in bonds:
            t = tuple((s[p] + e[p]) % lattice[p] for p in range(dim))
            ct = cl(t)
            if cs == ct:
                if cs == zero:
                    assert local(s) != local(t), "self-bond: lattice extent 1 along a bond axis"
                    H0 += embed(B, [local(s), local(t)], L)
            elif cs == zero:
                Hpair[lin(ct)] += embed(B, [local(s), L + local(t)], 2 * L)
            elif ct == zero:
                Hpair[lin(cs)] += embed(B, [L + local(s), local(t)], 2 * L)
    return dict(H0=H0, Hpair=Hpair, lattice=lattice, cluster=cluster, M=M, N=N, L=L, m=m, D=D,
                dim=dim)


def full_hamiltonian_apply(lattice, onsite, bonds):
    """Matrix-free action of the full-lattice Hamiltonian (Sec. 2.1, Eq. (TFI)/(AFH)) on a
    state vector of 2^n amplitudes, n = number of spins, site index row-major."""
    lattice = tuple(lattice)
    dim = len(lattice)
    sites = lattice_sites(lattice)
    index = {s: i for i, s in enumerate(sites)}
    n = len(sites)
    terms = []
    for s in sites:
        terms.append((onsite, (index[s],)))
        for e, B in bonds:
            t = tuple((s[p] + e[p]) % lattice[p] for p in range(dim))
            terms.append((B, (index[s], index[t])))
    return _apply_terms(terms, n), n


def _apply_terms(terms, n):
    """psi -> sum over (op, positions) of op acting on the spins `positions` of psi."""

    def apply(psi):
        psi = np.asarray(psi).reshape([2] * n)
        out = np.zeros_like(psi)
        for op, pos in terms:
            k = len(pos)
            if not np.any(op):
                continue
            o = op.reshape([2] * (2 * k))
            # contract the op's column indices with the state's axes `pos`
            moved = np.tensordot(o, psi, axes=(list(range(k, 2 * k)), list(pos)))
            # tensordot puts the op's row axes first; move them back to `pos`
            out += np.moveaxis(moved, list(range(k)), list(pos))
        return out.reshape(-1)

    return apply


def general_blocks(nspins, L, onsite, bonds):
    """Cluster blocks of a general spin-1/2 Hamiltonian (Sec. 2.1 pairwise form, Sec. 2.3
    cluster relaxation; no translation invariance), the input of Algorithm 5.

    Spins 0 .. nspins-1 are grouped into N = nspins / L clusters of L consecutive spins
    (cluster c holds spins c L .. c L + L - 1, in that factor order).  `onsite` is (nspins, 2, 2),
    one single-spin term per spin; `bonds` is a list of (s, t, B), B a 4 x 4 operator on the
    spins (s, t) with s the first factor.  A term inside one cluster goes to that cluster's
    H_i; a term between clusters i < j goes to H_ij, cluster i the first factor.

    Returns dict(Hi (N, m, m), Hij (K, D, D), pairs [(i, j)] for i < j in lexicographic order,
    N, L, m, D)."""
    assert nspins % L == 0 and nspins // L >= 2
    N = nspins // L
    m = 2 ** L
    D = m * m
    pairs = [(i, j) for i in range(N) for j in range(i + 1, N)]
    index = {pq: p for p, pq in enumerate(pairs)}
    Hi = np.zeros((N, m, m))
    Hij = np.zeros((len(pairs), D, D))
    for s in range(nspins):
        Hi[s // L] += embed(np.asarray(onsite[s]), [s % L], L)
    for s, t, B in bonds:
        cs, ct = s // L, t // L
        assert s != t
        if cs == ct:
            Hi[cs] += embed(np.asarray(B), [s % L, t % L], L)
        elif cs < ct:
            Hij[index[(cs, ct)]] += embed(np.asarray(B), [s % L, L + t % L], 2 * L)
        else:
            Hij[index[(ct, cs)]] += embed(np.asarray(B), [L + s % L, t % L], 2 * L)
    return dict(Hi=Hi, Hij=Hij, pairs=pairs, N=N, L=L, m=m, D=D)


def terms_apply(nspins, onsite, bonds):
    """Matrix-free action of sum_s onsite[s] + sum_(s,t,B) B on 2^nspins amplitudes."""
    terms = [(np.asarray(onsite[s]), (s,)) for s in range(nspins)]
    terms += [(np.asarray(B), (s, t)) for s, t, B in bonds]
    return _apply_terms(terms, nspins)


def exact_ground_energy_terms(nspins, onsite, bonds):
    """E_0 of a general spin Hamiltonian given as terms (as general_blocks), by exact
    diagonalisation (dense up to 10 spins, Lanczos above)."""
    apply = terms_apply(nspins, onsite, bonds)
    dim = 2 ** nspins
    if nspins <= 10:
        H = np.stack([apply(col) for col in np.eye(dim)], axis=1)
        return np.linalg.eigvalsh(H)[0]
    from scipy.sparse.linalg import LinearOperator, eigsh
    op = LinearOperator((dim, dim), matvec=apply, dtype=np.float64)
    return eigsh(op, k=1, which="SA", tol=1e-12, v0=np.ones(dim) / np.sqrt(dim))[0][0]


def exact_ground_energy(lattice, onsite, bonds, return_state=False):
    """Lowest eigenvalue E_0 of the full Hamiltonian, Eq. (groundstate), by exact
    diagonalisation: dense for <= 10 spins, Lanczos (scipy eigsh) above."""
    apply, n = full_hamiltonian_apply(lattice, onsite, bonds)
    dim = 2 ** n
    if n <= 10:
        H = np.stack([apply(col) for col in np.eye(dim)], axis=1)
        w, V = np.linalg.eigh(H)
        return (w[0], V[:, 0]) if return_state else w[0]
    from scipy.sparse.linalg import LinearOperator, eigsh
    op = LinearOperator((dim, dim), matvec=apply, dtype=np.float64)
    w, V = eigsh(op, k=1, which="SA", tol=1e-12, v0=np.ones(dim) / np.sqrt(dim))
    return (w[0], V[:, 0]) if return_state else w[0]


def tfim_chain_jw_energy(n, J, h):
    """Ground energy of the periodic TFI chain -h sum s^x - J sum s^z s^z (n >= 2 spins) by the
    Jordan-Wigner / Bogoliubov closed form: E_0 = -sum_k sqrt(J^2 + h^2 - 2 J h cos k) over the
    antiperiodic momenta k = (2j+1) pi / n, j = 0..n-1 (even-parity sector, which holds the
    ground state for J, h >= 0)."""
    k = (2 * np.arange(n) + 1) * np.pi / n
    return -np.sum(np.sqrt(J * J + h * h - 2 * J * h * np.cos(k)))
