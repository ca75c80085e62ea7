"""Algorithm 5 (general lattice, dense global matrix X) on a translation-invariant model,
for tiny lattices only.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  This is the un-reduced scheme that
Algorithm 6 specialises: every cluster i has its own rho_i, every pair i < j its own
rho~_ij, Lambda_ij, Lambda1_ij, Lambda2_ij, and the X step projects the full
(N D) x (N D) matrix X - eps G by one dense eigendecomposition.  It pins the translation-
invariant reduction, the block-DFT projection and the rho_0 update of ve_oracle against
the plain definitions.  Readings R1-R4, R7 of ve_oracle apply.
"""
import numpy as np

from .ve_oracle import (A1, A1_adj, A2, A2_adj, G_00, G_pair, T_inverse, eff_ham_0,
                        eff_ham_pair, neg_index, proj_psd)


def _lin(M, c):
    return int(np.ravel_multi_index(tuple(np.mod(c, M)), M))


def setup(pb):
    """Per-cluster and per-pair Hamiltonians of the full problem from the TI blocks:
    H_i = H_0, and H_ij (i first) = H_{0, j-i} (translation invariance, Sec. 3.3)."""
    M = np.array(pb.M)
    N, D = pb.N, pb.D
    coords = np.array(np.unravel_index(np.arange(N), tuple(M))).T
    Hfull = pb.model['Hpair']
    pairs, Hij = [], []
    for i in range(N):
        for j in range(i + 1, N):
            pairs.append((i, j))
            Hij.append(Hfull[_lin(tuple(M), coords[j] - coords[i])])
    return dict(pairs=pairs, Hij=np.array(Hij), coords=coords)


def initial_state(pb, s5):
    N, m, D = pb.N, pb.m, pb.D
    K = len(s5['pairs'])
    return dict(rho=np.broadcast_to(np.eye(m) / m, (N, m, m)).copy(),
                rt=np.broadcast_to(np.eye(D) / D, (K, D, D)).copy(),
                lam=np.zeros((K, D, D)), lam1=np.zeros((K, m, m)), lam2=np.zeros((K, m, m)),
                X=np.eye(N * D))


def iterate(pb, s5, st):
    """One sweep of Algorithm 5 (X step sign per reading R3)."""
    mu, nu, eps, N, m, D = pb.mu, pb.nu, pb.eps, pb.N, pb.m, pb.D
    pairs = s5['pairs']
    X = st['X']
    blk = lambda i, j: X[i * D:(i + 1) * D, j * D:(j + 1) * D]
    Hp_i = [eff_ham_0(pb.H0, blk(i, i)) for i in range(N)]
    Hp_ij = np.array([eff_ham_pair(s5['Hij'][p], blk(i, j)) for p, (i, j) in enumerate(pairs)])
    rho_i = st['rho']
    first = np.array([rho_i[i] for i, j in pairs])
    second = np.array([rho_i[j] for i, j in pairs])
    rhs = (mu * st['rt'] + A1_adj(nu * first - st['lam1']) + A2_adj(nu * second - st['lam2'])
           + st['lam'] - Hp_ij)
    rho = T_inverse(rhs, mu, nu)
    rt = proj_psd(rho - st['lam'] / mu)
    new_rho_i = np.empty_like(rho_i)
    a1, a2 = A1(rho), A2(rho)
    for i in range(N):
        acc = -Hp_i[i]
        for p, (a, b) in enumerate(pairs):
            if a == i:
                acc = acc + nu * a1[p] + st['lam1'][p]
            if b == i:
                acc = acc + nu * a2[p] + st['lam2'][p]
        r = acc / (nu * (N - 1))
        new_rho_i[i] = r + (1.0 - np.trace(r)) / m * np.eye(m)
    first = np.array([new_rho_i[i] for i, j in pairs])
    second = np.array([new_rho_i[j] for i, j in pairs])
    lam = st['lam'] + mu * (rt - rho)
    lam1 = st['lam1'] + nu * (a1 - first)
    lam2 = st['lam2'] + nu * (a2 - second)
    G = np.zeros((N * D, N * D))
    for i in range(N):
        G[i * D:(i + 1) * D, i * D:(i + 1) * D] = G_00(new_rho_i[i])
    for p, (i, j) in enumerate(pairs):
        g = G_pair(rho[p])
        G[i * D:(i + 1) * D, j * D:(j + 1) * D] = g
        G[j * D:(j + 1) * D, i * D:(i + 1) * D] = g.T
    Xn = proj_psd(X - eps * G)
    st.update(rho=new_rho_i, rt=rt, lam=lam, lam1=lam1, lam2=lam2, X=Xn)


def ti_view(pb, s5, st):
    """The Algorithm-6 variables read off the Algorithm-5 state: rho_0, and for delta != 0
    the pair (0, delta) with its multipliers, plus X's first block row."""
    N, D = pb.N, pb.D
    index = {pq: p for p, pq in enumerate(s5['pairs'])}
    slots = [index[(0, j)] for j in range(1, N)]
    return dict(rho0=st['rho'][0], rt=st['rt'][slots], lam=st['lam'][slots],
                lam1=st['lam1'][slots], lam2=st['lam2'][slots],
                X=np.array([st['X'][0:D, j * D:(j + 1) * D] for j in range(N)]))


__all__ = ['setup', 'initial_state', 'iterate', 'ti_view', 'neg_index']
