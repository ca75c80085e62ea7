"""Algorithm 5 (general lattice, dense global matrix X) of Khoo & Lindsey, arXiv:2106.02682,
Sec. 3.2 "Practical scheme": every cluster i has its own rho_i and H_i, every pair i < j its own
H_ij, rho~_ij, Lambda_ij, Lambda1_ij, Lambda2_ij, and the X step projects the full (N D) x (N D)
matrix X - eps G by one dense eigendecomposition.  No translation invariance is assumed.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Two uses:
  * the parity reference of the general (non-translation-invariant) GPU solver;
  * on a translation-invariant model (setup), the un-reduced scheme that Algorithm 6 specialises,
    which pins the block-DFT projection and the rho_0 update of ve_oracle.
Readings R1-R4, R7 and R8 of ve_oracle apply; R8 (convergence measures) becomes
  energy per spin  E = (sum_i Tr[H_i rho_i] + sum_{i<j} Tr[H_ij rho_ij]) / (N L),
  Eq. (feasErr)    sqrt(sum_{i<j} (|A1 rho_ij - rho_i|^2 + |A2 rho_ij - rho_j|^2
                                   + |rho_ij - rho~_ij|^2) / K),  K = N (N - 1) / 2,
which on a translation-invariant state equal the Algorithm-6 measures.
"""
import numpy as np

from .ve_oracle import (A1, A1_adj, A2, A2_adj, G_00, G_pair, T_inverse, eff_ham_0,
                        eff_ham_pair, neg_index, proj_psd)


class GeneralProblem:
    """An Algorithm-5 instance from cluster blocks (models.general_blocks, or
    fermions.fermion_blocks): N clusters of L sites, H_i (N, m, m), H_ij (K, D, D) for the pairs
    i < j in lexicographic order.  fermionic=True takes the global matrix of Eq. (sdpFerm):
    its off-diagonal blocks carry the parity signs of fermions.parity_signs (the diagonal blocks
    and the partial traces are the spin ones)."""

    def __init__(self, blocks, mu=10.0, nu=10.0, eps=2.0, fermionic=False):
        self.N, self.L, self.m, self.D = blocks['N'], blocks['L'], blocks['m'], blocks['D']
        self.mu, self.nu, self.eps = float(mu), float(nu), float(eps)
        self.sign = None
        if fermionic:
            from .fermions import parity_signs
            self.sign = parity_signs(self.m)
        assert self.N >= 2


def _G_pair(pb, rho):
    """Off-diagonal blocks of the global matrix (with the fermionic parity signs if any)."""
    sign = getattr(pb, 'sign', None)   # translation-invariant problems carry none
    g = G_pair(rho)
    return g if sign is None else sign * g


def _eff_ham_pair(pb, H, Xij):
    """H'_ij of Eq. (effHam): H minus the adjoint of the off-diagonal G map applied to X_ij (and
    its transpose); the signed map's adjoint applies the same signs to X first."""
    sign = getattr(pb, 'sign', None)
    return eff_ham_pair(H, Xij if sign is None else sign * Xij)


def general_setup(blocks):
    return dict(pairs=list(blocks['pairs']), Hi=np.array(blocks['Hi']),
                Hij=np.array(blocks['Hij']))


def _lin(M, c):
    return int(np.ravel_multi_index(tuple(np.mod(c, M)), M))


def setup(pb):
    """Per-cluster and per-pair Hamiltonians of a translation-invariant problem (ve_oracle
    Problem) from its blocks: H_i = H_0, and H_ij (i first) = H_{0, j-i} (Sec. 3.3)."""
    M = np.array(pb.M)
    N = pb.N
    coords = np.array(np.unravel_index(np.arange(N), tuple(M))).T
    Hfull = pb.model['Hpair']
    pairs, Hij = [], []
    for i in range(N):
        for j in range(i + 1, N):
            pairs.append((i, j))
            Hij.append(Hfull[_lin(tuple(M), coords[j] - coords[i])])
    return dict(pairs=pairs, Hij=np.array(Hij), Hi=np.broadcast_to(pb.H0, (N,) + pb.H0.shape),
                coords=coords)


def initial_state(pb, s5):
    """Reading R7 of ve_oracle: Lambdas = 0, rho_i = I/m, rho~_ij = I/D, X = I."""
    N, m, D = pb.N, pb.m, pb.D
    K = len(s5['pairs'])
    return dict(rho=np.broadcast_to(np.eye(m) / m, (N, m, m)).copy(),
                rt=np.broadcast_to(np.eye(D) / D, (K, D, D)).copy(),
                lam=np.zeros((K, D, D)), lam1=np.zeros((K, m, m)), lam2=np.zeros((K, m, m)),
                X=np.eye(N * D), energy=np.nan, it=0)


def _pair_index(s5):
    p = np.array(s5['pairs'], dtype=np.int64).reshape(-1, 2)
    return p[:, 0], p[:, 1]


def pair_blocks(X, N, D, pi, pj):
    """The blocks X_ij (K, D, D) of the dense N D x N D matrix X for the pairs (pi, pj)."""
    return X.reshape(N, D, N, D)[pi, :, pj, :]


def iterate(pb, s5, st):
    """One sweep of Algorithm 5 (X step sign per reading R3).  Updates `st` in place and
    returns dict(energy, feas_err, d_energy, residual)."""
    mu, nu, eps, N, m, D, L = pb.mu, pb.nu, pb.eps, pb.N, pb.m, pb.D, pb.L
    pi, pj = _pair_index(s5)
    K = len(pi)
    X = st['X']
    # effective Hamiltonians, Eq. (effHam)
    Hp_i = [eff_ham_0(s5['Hi'][i], X[i * D:(i + 1) * D, i * D:(i + 1) * D]) for i in range(N)]
    Hp_ij = _eff_ham_pair(pb, s5['Hij'], pair_blocks(X, N, D, pi, pj))
    # closed-form pair update, Eq. (rhoijUpdate)
    rho_i = st['rho']
    rhs = (mu * st['rt'] + A1_adj(nu * rho_i[pi] - st['lam1'])
           + A2_adj(nu * rho_i[pj] - st['lam2']) + st['lam'] - Hp_ij)
    rho = T_inverse(rhs, mu, nu)
    # Eq. (rhoijTildeUpdate)
    rt = proj_psd(rho - st['lam'] / mu)
    # one-cluster marginals, Eq. (rhoiUpdate): pairs (i, j > i) through A1, (j < i, i) via A2
    a1, a2 = A1(rho), A2(rho)
    acc = -np.array(Hp_i)
    np.add.at(acc, pi, nu * a1 + st['lam1'])
    np.add.at(acc, pj, nu * a2 + st['lam2'])
    r = acc / (nu * (N - 1))
    z = (1.0 - np.einsum('nii->n', r)) / m
    new_rho_i = r + z[:, None, None] * np.eye(m)
    # dual updates
    lam = st['lam'] + mu * (rt - rho)
    lam1 = st['lam1'] + nu * (a1 - new_rho_i[pi])
    lam2 = st['lam2'] + nu * (a2 - new_rho_i[pj])
    # global matrix G[{rho_i}, {rho_ij}] (Sec. 2.2) and the X step
    G4 = np.zeros((N, N, D, D))
    g = _G_pair(pb, rho)
    G4[pi, pj] = g
    G4[pj, pi] = np.swapaxes(g, 1, 2)
    for i in range(N):
        G4[i, i] = G_00(new_rho_i[i])
    G = G4.transpose(0, 2, 1, 3).reshape(N * D, N * D)
    Xn = proj_psd(X - eps * G)
    # convergence measures (R8 of ve_oracle, general form)
    energy = (np.einsum('nij,nji->', s5['Hi'], new_rho_i)
              + np.einsum('pij,pji->', s5['Hij'], rho)) / (N * L)
    feas = np.sqrt((np.sum((a1 - new_rho_i[pi]) ** 2) + np.sum((a2 - new_rho_i[pj]) ** 2)
                    + np.sum((rho - rt) ** 2)) / K)
    d_energy = abs(energy - st['energy']) if np.isfinite(st['energy']) else np.inf
    st.update(rho=new_rho_i, rt=rt, lam=lam, lam1=lam1, lam2=lam2, X=Xn, energy=energy,
              it=st['it'] + 1)
    return dict(energy=energy, feas_err=feas, d_energy=d_energy, residual=max(feas, d_energy))


def run(pb, s5, st, iters, tol=0.0, check_every=10):
    diag = None
    for t in range(iters):
        diag = iterate(pb, s5, st)
        if tol > 0 and (t + 1) % check_every == 0 and diag['residual'] <= tol:
            break
    return diag


def certified_bound(pb, s5, st):
    """Lower bound on E_0 (per spin) of the general problem, valid for ANY multipliers and PSD X.

    For X >= 0, E_0 >= F[X] (Eq. (partialDual)).  Adding <Lambda1_ij, A1 rho_ij - rho_i> +
    <Lambda2_ij, A2 rho_ij - rho_j> (zero on the feasible set; the sign of the Lagrangian terms
    whose minimisation gives Eq. (rhoijUpdate)) to the objective and using rho >= 0, Tr = 1:
        F[X] >= sum_i lmin(K_i) + sum_{i<j} lmin(K_ij),
        K_ij = H'_ij + A1^* Lambda1_ij + A2^* Lambda2_ij,
        K_i  = H'_i - sum_{j>i} Lambda1_ij - sum_{j<i} Lambda2_ji.
    X is PSD only up to rounding: X + s I with s = max(0, -lmin(X)) is PSD and lowers every H'_i
    by s m I (the adjoint of G_00 maps I to m I), hence the correction N m s.
    Returns dict(bound_per_spin, raw_bound, x_min_eig, x_neg_correction, primal_per_spin)."""
    N, m, D, L = pb.N, pb.m, pb.D, pb.L
    pi, pj = _pair_index(s5)
    X = st['X']
    Kp = (_eff_ham_pair(pb, s5['Hij'], pair_blocks(X, N, D, pi, pj)) + A1_adj(st['lam1'])
          + A2_adj(st['lam2']))
    Ki = np.array([eff_ham_0(s5['Hi'][i], X[i * D:(i + 1) * D, i * D:(i + 1) * D])
                   for i in range(N)])
    np.subtract.at(Ki, pi, st['lam1'])
    np.subtract.at(Ki, pj, st['lam2'])
    raw = float(np.sum(np.linalg.eigvalsh(Ki)[:, 0]) + np.sum(np.linalg.eigvalsh(Kp)[:, 0]))
    xmin = float(np.linalg.eigvalsh(X)[0])
    corr = N * m * max(0.0, -xmin)
    return dict(bound_per_spin=(raw - corr) / (N * L), raw_bound=raw, x_min_eig=xmin,
                x_neg_correction=corr, primal_per_spin=st['energy'])


def pack_state(pb, s5, st):
    """rho_i (N m^2), rho~ (K D^2), Lambda (K D^2), Lambda1 (K m^2), Lambda2 (K m^2),
    X (N D x N D), each row-major, as one float64 vector."""
    return np.concatenate([st['rho'].ravel(), st['rt'].ravel(), st['lam'].ravel(),
                           st['lam1'].ravel(), st['lam2'].ravel(), st['X'].ravel()])


def unpack_state(pb, s5, vec, energy=np.nan, it=0):
    N, m, D = pb.N, pb.m, pb.D
    K = len(s5['pairs'])
    sizes = [N * m * m, K * D * D, K * D * D, K * m * m, K * m * m, (N * D) ** 2]
    parts = np.split(np.asarray(vec, dtype=np.float64), np.cumsum(sizes)[:-1])
    return dict(rho=parts[0].reshape(N, m, m).copy(), rt=parts[1].reshape(K, D, D).copy(),
                lam=parts[2].reshape(K, D, D).copy(), lam1=parts[3].reshape(K, m, m).copy(),
                lam2=parts[4].reshape(K, m, m).copy(), X=parts[5].reshape(N * D, N * D).copy(),
                energy=energy, it=it)


def ti_view(pb, s5, st):
    """The Algorithm-6 variables read off the Algorithm-5 state: rho_0, and for delta != 0
    the pair (0, delta) with its multipliers, plus X's first block row."""
    N, D = pb.N, pb.D
    index = {pq: p for p, pq in enumerate(s5['pairs'])}
    slots = [index[(0, j)] for j in range(1, N)]
    return dict(rho0=st['rho'][0], rt=st['rt'][slots], lam=st['lam'][slots],
                lam1=st['lam1'][slots], lam2=st['lam2'][slots],
                X=np.array([st['X'][0:D, j * D:(j + 1) * D] for j in range(N)]))


__all__ = ['GeneralProblem', 'general_setup', 'setup', 'initial_state', 'iterate', 'run',
           'certified_bound', 'pack_state', 'unpack_state', 'ti_view', 'neg_index']
