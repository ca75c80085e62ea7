"""Plain CPU FP64 oracle for the translation-invariant ADMM / projected dual-gradient ascent
of Khoo & Lindsey, "Scalable semidefinite programming approach to variational embedding for
quantum many-body problems" (arXiv:2106.02682), Algorithm 6, with its convergence measures
(Sec. 4, Eq. (feasErr)) and a certified dual lower bound derived from Sec. 2.4 / Sec. 3.1.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
reference legs may import this module.  The GPU solver never imports, links or calls it, and
the two share no code.  Every step is written the slow, obvious way: numpy einsum for index
maps, numpy.linalg.eigh as the eigensolver step, numpy.fft as the DFT step.

Notation: m = 2^L (cluster dimension), D = m^2 (pair dimension and X-block size), N clusters
(= number of wavevectors), P = N - 1 pair offsets delta != 0.  Pair arrays are indexed by
delta's linear index minus one; X blocks by delta's linear index (X[0] = X_{0,0}).

Readings of the paper (where it is silent, ambiguous or garbled):
  R1  Operator collection: the complete, orthonormal matrix-unit basis O_(a,b) = E_ab,
      n_i = m^2 (Sec. 2.2: "complete operator collection").  Then
      G_{0,d}[rho]_{(a,b),(c,d')} = Tr[(E_ba (x) E_cd') rho] = rho_{(a,d'),(b,c)}  (a realignment)
      G_{0,0}[rho0]_{(a,b),(c,d')} = Tr[E_ba E_cd' rho0] = delta_ac rho0_{d',b}.
  R2  Eq. (effHam) reads "H_ij[X_ij] := H_i - ..." and "O_{i,alpha}^dag (x) O_{i,beta}"; we
      read H_ij - [sum conj(X)_ab O_{i,a}^dag (x) O_{j,b} + h.c.], the form that makes
      Tr[H'_ij rho_ij] = Tr[H_ij rho_ij] - 2 <X_ij, G_ij[rho_ij]> (the Lagrangian term -Tr[XG]).
  R3  X step sign.  Algorithms 1, 5 and 6 write X <- Pi(X + eps G).  With Eq. (effHam) and
      Eq. (gradX) (grad_X F = -G) ascent on F is X <- Pi(X - eps G); that is the only sign whose
      fixed point satisfies the KKT conditions (G >= 0, <X, G> = 0).  We take X - eps G.
  R4  The rho_0 update divides by nu (N - 1) with N the total number of clusters (the sum in
      Eq. (rhoiUpdate) runs over all other clusters), although Sec. 3.3 reuses M for the
      clusters per axis.
  R5  Pi_{>=0} (Sec. 3, written with "min" for "argmin") is applied to the complex Hermitian
      blocks X^_k (X_{0,-d} = X_{0,d}^T makes them Hermitian, not real): Hermitian eigen-
      decomposition, negative eigenvalues set to zero.
  R6  The DFT in Algorithm 6 is unitary (1/sqrt(N) both ways) and its inverse sum runs over k
      (the printed index "j" is a typo).  The oracle uses the unitary pair exactly.
  R7  Initialisation (Sec. 4): Lambda = Lambda1 = Lambda2 = 0, rho_0 = I/m, rho~ = I/D, X = I.
  R8  Convergence measures: per-spin energy E = (Tr[H_0 rho_0] + 1/2 sum_d Tr[H_{0,d} rho_{0,d}])/L
      with the bare H and the rho_{0,d} of the closed-form update; Eq. (feasErr) with the new
      rho_0 and rho~; residual r = max(feasErr, |E - E_prev|).
"""
import numpy as np

from . import models  # noqa: F401  (re-exported for callers: oracle.ve_oracle.models)


# ----------------------------------------------------------------------------------------
# Linear maps of Sec. 2.2 / 3.1 on D x D pair operators (cluster 0 = first tensor factor)
# ----------------------------------------------------------------------------------------

def _split(A):
    """View the trailing (D, D) axes as (m, m, m, m): [a, b, c, d] = A[(a,b),(c,d)]."""
    D = A.shape[-1]
    m = int(round(np.sqrt(D)))
    return A.reshape(A.shape[:-2] + (m, m, m, m)), m


def A1(rho):
    """A_1 = Tr_{2}: partial trace over the second cluster (Sec. 3.1, Eq. (sdpC2))."""
    r, m = _split(rho)
    return np.einsum('...abcb->...ac', r)


def A2(rho):
    """A_2 = Tr_{1}: partial trace over the first cluster (Sec. 3.1, Eq. (sdpC2))."""
    r, m = _split(rho)
    return np.einsum('...abad->...bd', r)


def A1_adj(Y):
    """A_1^*: Y -> Y (x) I_m, the Frobenius adjoint of Tr_{2}."""
    m = Y.shape[-1]
    return np.einsum('...ac,bd->...abcd', Y, np.eye(m)).reshape(Y.shape[:-2] + (m * m, m * m))


def A2_adj(Y):
    """A_2^*: Y -> I_m (x) Y, the Frobenius adjoint of Tr_{1}."""
    m = Y.shape[-1]
    return np.einsum('ac,...bd->...abcd', np.eye(m), Y).reshape(Y.shape[:-2] + (m * m, m * m))


def G_pair(rho):
    """Off-diagonal block of the global matrix, Sec. 2.2: G_{0,d}[rho]_{ab} =
    Tr[(O_a^dag (x) O_b) rho]; with matrix units (reading R1) entry (a,b),(c,d) = rho_{(a,d),(b,c)}."""
    r, m = _split(rho)
    return np.einsum('...adbc->...abcd', r).reshape(rho.shape)


def G_pair_adj(X):
    """Frobenius adjoint of G_pair: entry (p,q),(r,s) = X_{(p,r),(s,q)}.  Since
    Tr[S rho] = <S^T, rho>_F, the operator sum_{ab} X_{ab} O_a^dag (x) O_b of Eq. (effHam) is the
    TRANSPOSE of this adjoint; eff_ham_pair adds both, so either serves there."""
    x, m = _split(X)
    return np.einsum('...prsq->...pqrs', x).reshape(X.shape)


def G_00(rho0):
    """Diagonal block of the global matrix, Sec. 2.2: (G_00)_{ab} = Tr[O_a^dag O_b rho0];
    with matrix units entry (a,b),(c,d) = delta_ac rho0_{d,b}."""
    m = rho0.shape[-1]
    return np.einsum('ac,db->abcd', np.eye(m), rho0).reshape(m * m, m * m)


def G_00_adj(X00):
    """Frobenius adjoint of G_00: sum_{ab} X_{ab} O_a^dag O_b, entry (b,d) = sum_a X_{(a,b),(a,d)}."""
    x, m = _split(X00)
    return np.einsum('abad->bd', x)


def eff_ham_0(H0, X00):
    """H_0[X_00] of Eq. (effHam) (real case, conj(X) = X)."""
    return H0 - G_00_adj(X00)


def eff_ham_pair(H, X):
    """H_{0,d}[X_{0,d}] of Eq. (effHam) with the h.c. term (reading R2)."""
    S = G_pair_adj(X)
    return H - (S + np.swapaxes(S, -1, -2))


def T_inverse(Y, mu, nu):
    """(mu + nu A1^* A1 + nu A2^* A2)^{-1} Y, the solve in Eq. (rhoijUpdate).

    A1^*A1 = m P1 and A2^*A2 = m P2 with P1 Y = Tr_2(Y) (x) I / m, P2 Y = I (x) Tr_1(Y) / m the
    Frobenius-orthogonal projectors; they commute with P1 P2 = Q, Q Y = Tr(Y) I / D.  On the
    ranges of (1 - P1 - P2 + Q), (P1 - Q) + (P2 - Q) and Q the operator acts as mu, mu + nu m
    and mu + 2 nu m, so its inverse is the sum of those projectors over those values.
    """
    D = Y.shape[-1]
    m = int(round(np.sqrt(D)))
    a = nu * m
    P1 = A1_adj(A1(Y)) / m
    P2 = A2_adj(A2(Y)) / m
    Q = np.einsum('...ii->...', Y)[..., None, None] * np.eye(D) / D
    return (Y - P1 - P2 + Q) / mu + (P1 + P2 - 2 * Q) / (mu + a) + Q / (mu + 2 * a)


def _proj_psd_one_thread(C):
    w, V = np.linalg.eigh(C)
    return (V * np.maximum(w, 0.0)[..., None, :]) @ np.conj(np.swapaxes(V, -1, -2))


# Optional thread pool over the independent matrices of a batch (the pair offsets delta and the
# wavevectors k of one sweep).  Every matrix still goes through the same eigh call on its own,
# so the results do not depend on the number of threads; numpy releases the GIL inside LAPACK.
_POOL = None
_THREADS = 1


def set_threads(n):
    """Run the batched projections of a sweep on n host threads (1: no pool)."""
    global _POOL, _THREADS
    import concurrent.futures
    if _POOL is not None:
        _POOL.shutdown()
        _POOL = None
    _THREADS = max(1, int(n))
    if _THREADS > 1:
        _POOL = concurrent.futures.ThreadPoolExecutor(max_workers=_THREADS)


def proj_psd(C):
    """Pi_{>=0}(C) (Sec. 3): nearest PSD matrix in Frobenius norm = eigendecomposition with
    negative eigenvalues set to zero.  Works batched, real symmetric or complex Hermitian
    (reading R5)."""
    if _POOL is None or C.ndim < 3 or C.shape[0] < 2 * _THREADS:
        return _proj_psd_one_thread(C)
    parts = list(_POOL.map(_proj_psd_one_thread, np.array_split(C, _THREADS)))
    return np.concatenate(parts)


# ----------------------------------------------------------------------------------------
# Translation-invariant solver state and one sweep of Algorithm 6
# ----------------------------------------------------------------------------------------

class Problem:
    """A translation-invariant instance: cluster blocks (see models.cluster_model) plus the
    algorithm parameters mu, nu, eps (Sec. 4 uses mu = nu = 10, eps = 2)."""

    def __init__(self, model, mu=10.0, nu=10.0, eps=2.0):
        self.model = model
        self.H0 = model['H0']
        self.Hpair = model['Hpair'][1:]            # (P, D, D), pair slot = linear index - 1
        self.M = model['M']
        self.N, self.L, self.m, self.D = model['N'], model['L'], model['m'], model['D']
        self.mu, self.nu, self.eps = float(mu), float(nu), float(eps)
        assert self.N >= 2


def initial_state(pb):
    """Initial variables of Sec. 4 (reading R7)."""
    N, m, D = pb.N, pb.m, pb.D
    P = N - 1
    X = np.zeros((N, D, D))
    X[0] = np.eye(D)
    return dict(rho0=np.eye(m) / m,
                rt=np.broadcast_to(np.eye(D) / D, (P, D, D)).copy(),
                lam=np.zeros((P, D, D)), lam1=np.zeros((P, m, m)), lam2=np.zeros((P, m, m)),
                X=X, energy=np.nan, it=0)


def _lattice_dft(blocks, M, inverse):
    """Unitary d-dimensional DFT over the cluster-offset axes of a first block row
    (Sec. 3.3): forward X^_k = N^{-1/2} sum_j exp(-i 2 pi j.k / M) X_j, inverse with +i."""
    arr = blocks.reshape(tuple(M) + blocks.shape[1:])
    axes = tuple(range(len(M)))
    f = np.fft.ifftn if inverse else np.fft.fftn
    out = f(arr, axes=axes, norm='ortho')
    return out.reshape(blocks.shape)


def iterate(pb, st):
    """One sweep of Algorithm 6.  Updates `st` in place and returns the diagnostics of
    reading R8: dict(energy, feas_err, d_energy, residual)."""
    mu, nu, eps, N, m, L = pb.mu, pb.nu, pb.eps, pb.N, pb.m, pb.L
    X = st['X']
    # effective Hamiltonians from the current X (Algorithm 6, first two updates)
    H0p = eff_ham_0(pb.H0, X[0])
    Hp = eff_ham_pair(pb.Hpair, X[1:])
    # closed-form pair update, Eq. (rhoijUpdate)
    rhs = (mu * st['rt'] + A1_adj(nu * st['rho0'] - st['lam1'])
           + A2_adj(nu * st['rho0'] - st['lam2']) + st['lam'] - Hp)
    rho = T_inverse(rhs, mu, nu)
    # projection of the shifted pair marginals, Eq. (rhoijTildeUpdate)
    rt = proj_psd(rho - st['lam'] / mu)
    # one-cluster marginal, Eq. (rhoiUpdate) in translation-invariant form (reading R4)
    rho0p = (np.sum(nu * A1(rho) + st['lam1'], axis=0) - H0p) / (nu * (N - 1))
    z = (1.0 - np.trace(rho0p)) / m
    rho0 = rho0p + z * np.eye(m)
    # dual updates (Algorithm 4 / 6)
    lam = st['lam'] + mu * (rt - rho)
    lam1 = st['lam1'] + nu * (A1(rho) - rho0)
    lam2 = st['lam2'] + nu * (A2(rho) - rho0)
    # global step on X (reading R3 for the sign), block DFT, per-k projection, inverse DFT
    Xp = np.empty_like(X)
    Xp[0] = X[0] - eps * G_00(rho0)
    Xp[1:] = X[1:] - eps * G_pair(rho)
    Xhat = _lattice_dft(Xp, pb.M, inverse=False)
    Yk = proj_psd(Xhat)
    Xnew = np.real(_lattice_dft(Yk, pb.M, inverse=True))
    # convergence measures (reading R8)
    energy = (np.trace(pb.H0 @ rho0)
              + 0.5 * np.einsum('pij,pji->', pb.Hpair, rho)) / L
    feas = np.sqrt((np.sum((A1(rho) - rho0) ** 2) + np.sum((A2(rho) - rho0) ** 2)
                    + np.sum((rho - rt) ** 2)) / (N - 1))
    d_energy = abs(energy - st['energy']) if np.isfinite(st['energy']) else np.inf
    st.update(rho0=rho0, rt=rt, lam=lam, lam1=lam1, lam2=lam2, X=Xnew, energy=energy,
              it=st['it'] + 1, rho=rho)
    return dict(energy=energy, feas_err=feas, d_energy=d_energy,
                residual=max(feas, d_energy))


def run(pb, st, iters, tol=0.0, check_every=10):
    """Iterate until `iters` sweeps or residual <= tol, tested every `check_every` sweeps."""
    diag = None
    for t in range(iters):
        diag = iterate(pb, st)
        if tol > 0 and (t + 1) % check_every == 0 and diag['residual'] <= tol:
            break
    return diag


# ----------------------------------------------------------------------------------------
# Certified lower bound (derived from weak duality of Eq. (partialDual) and Eq. (lagrangian))
# ----------------------------------------------------------------------------------------

def lattice_offsets(M):
    """All cluster offsets in linear-index order (row-major)."""
    return np.array(np.unravel_index(np.arange(int(np.prod(M))), M)).T


def neg_index(M):
    """Linear index of -delta for every linear index delta."""
    offs = lattice_offsets(M)
    neg = (-offs) % np.array(M)
    return np.ravel_multi_index(tuple(neg.T), M)


def pair_counts(M):
    """c(delta) = #{clusters a : l(a) < l(a + delta)}, l = row-major linear index: the number
    of ordered pairs a < b of Algorithm 5 that Algorithm 6 represents by rho_{0,delta}."""
    M = tuple(M)
    N = int(np.prod(M))
    offs = lattice_offsets(M)
    c = np.zeros(N, dtype=np.int64)
    for a in range(N):
        b = np.ravel_multi_index(tuple(((offs[a] + offs) % np.array(M)).T), M)
        c += (b > a)
    return c


def certified_bound(pb, st):
    """Lower bound on E_0 (per spin) valid for ANY multipliers Lambda1, Lambda2 and PSD X.

    For X >= 0, E_0 >= E_0^(2) >= F[X] (Eq. (partialDual)).  For the pair (a, b), a < b, with
    offset delta = b - a take multipliers Lambda1_delta (first factor) and Lambda1_{-delta}
    (second factor).  Adding <L1, A1 rho_ab - rho_a> + <L2, A2 rho_ab - rho_b> (zero on the
    feasible set) and using rho >= 0, Tr = 1 gives
        F[X] >= N lmin(K_0) + sum_delta c(delta) lmin(K_delta),
        K_delta = H'_{0,delta} + A1^* Lambda1_delta + A2^* Lambda1_{-delta},
        K_0     = H'_0 - sum_delta Lambda1_delta.
    The stored X is PSD only up to rounding: with lambda_X = min_k lmin(C_k), C_k the
    unnormalised block DFT (the eigen-blocks of the block-circulant X), X + s I with
    s = max(0, -lambda_X) is PSD and lowers every H'_0 by s m I, hence the correction N m s.
    Returns dict(bound_per_spin, raw_bound, x_min_eig, x_neg_correction, primal_per_spin).
    """
    N, m, L = pb.N, pb.m, pb.L
    X = st['X']
    lam1 = st['lam1']
    neg = neg_index(pb.M)                      # over linear indices 0..N-1
    lam1_neg = lam1[neg[1:] - 1]              # Lambda1_{-delta} for delta = 1..N-1
    K = (eff_ham_pair(pb.Hpair, X[1:]) + A1_adj(lam1) + A2_adj(lam1_neg))
    K0 = eff_ham_0(pb.H0, X[0]) - np.sum(lam1, axis=0)
    lmin_pairs = np.linalg.eigvalsh(K)[:, 0]
    lmin0 = np.linalg.eigvalsh(K0)[0]
    c = pair_counts(pb.M)[1:]
    raw = N * lmin0 + float(np.sum(c * lmin_pairs))
    Chat = _lattice_dft(X, pb.M, inverse=False) * np.sqrt(N)   # unnormalised eigen-blocks
    xmin = float(np.min(np.linalg.eigvalsh(Chat)[:, 0]))
    corr = N * m * max(0.0, -xmin)
    return dict(bound_per_spin=(raw - corr) / (N * L), raw_bound=raw, x_min_eig=xmin,
                x_neg_correction=corr, primal_per_spin=st['energy'])


# ----------------------------------------------------------------------------------------
# Packed state (the interchange layout also used by the solver library's get/set state)
# ----------------------------------------------------------------------------------------

def pack_state(pb, st):
    """Concatenate rho0 (m^2), rho~ (P D^2), Lambda (P D^2), Lambda1 (P m^2), Lambda2 (P m^2),
    X (N D^2) as one float64 vector, each block row-major."""
    return np.concatenate([st['rho0'].ravel(), st['rt'].ravel(), st['lam'].ravel(),
                           st['lam1'].ravel(), st['lam2'].ravel(), st['X'].ravel()])


def unpack_state(pb, vec, energy=np.nan, it=0):
    N, m, D = pb.N, pb.m, pb.D
    P = N - 1
    sizes = [m * m, P * D * D, P * D * D, P * m * m, P * m * m, N * D * D]
    parts = np.split(np.asarray(vec, dtype=np.float64), np.cumsum(sizes)[:-1])
    return dict(rho0=parts[0].reshape(m, m).copy(), rt=parts[1].reshape(P, D, D).copy(),
                lam=parts[2].reshape(P, D, D).copy(), lam1=parts[3].reshape(P, m, m).copy(),
                lam2=parts[4].reshape(P, m, m).copy(), X=parts[5].reshape(N, D, D).copy(),
                energy=energy, it=it)
