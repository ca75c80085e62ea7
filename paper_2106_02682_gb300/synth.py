"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU oracle's callers.

Only random-matrix and workload generators live here (no step of the solver's arithmetic):
  * symmetric_batch / hermitian_batch: matrices shaped like the projection inputs
    rho - Lambda/mu and the wavevector blocks -- O(1) entries, eigenvalues of both signs, plus a
    share with repeated eigenvalues and low rank, which stress the eigensolvers;
  * circulant_first_row: a first block row X_{0,delta} obeying X_{0,-delta} = X_{0,delta}^T, the
    structure of the dual matrix in Algorithm 6;
  * workloads: the named benchmark instances (lattice, cluster, field) used by bench.py;
  * batch_instances: seeded families of independent instances for batched runs;
  * disordered_chain: a general (not translation-invariant) spin chain as a list of terms, the
    input of the general solver: random fields and long-range random couplings;
  * fermion_ring: the spinless-fermion ring of the paper's fermionic section as hopping and
    density-density terms.
The default seed is 20210604.
"""
import numpy as np

SEED = 20210604


def _rng(seed):
    return np.random.default_rng(SEED if seed is None else SEED + int(seed))


def symmetric_batch(count, n, seed=None):
    rng = _rng(seed)
    A = rng.normal(size=(count, n, n))
    A = 0.5 * (A + np.swapaxes(A, 1, 2))
    # every 7th matrix: repeated eigenvalues (+1 / -1 / 0 blocks) in a random orthogonal basis
    for b in range(0, count, 7):
        Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
        lam = np.repeat(np.array([1.0, -1.0, 0.0]), (n + 2) // 3)[:n]
        A[b] = (Q * lam) @ Q.T
    return A


def hermitian_batch(count, n, seed=None):
    rng = _rng(seed)
    A = rng.normal(size=(count, n, n)) + 1j * rng.normal(size=(count, n, n))
    A = 0.5 * (A + np.conj(np.swapaxes(A, 1, 2)))
    for b in range(0, count, 7):
        Z = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        Q, _ = np.linalg.qr(Z)
        lam = np.repeat(np.array([1.0, -1.0, 0.0]), (n + 2) // 3)[:n]
        A[b] = (Q * lam) @ np.conj(Q.T)
    return A


def neg_linear_index(M):
    """Row-major linear index of -delta for every cluster offset delta of the lattice M."""
    M = tuple(int(x) for x in M)
    idx = np.arange(int(np.prod(M)))
    coords = np.array(np.unravel_index(idx, M))
    neg = (-coords) % np.array(M)[:, None]
    return np.ravel_multi_index(tuple(neg), M)


def circulant_first_row(M, D, seed=None):
    """Random N x D x D first block row with X_{0,-delta} = X_{0,delta}^T and a diagonal shift
    that leaves the block-circulant matrix indefinite (both signs to project)."""
    rng = _rng(seed)
    N = int(np.prod(M))
    X = rng.normal(size=(N, D, D)) / np.sqrt(N)
    neg = neg_linear_index(M)
    X = 0.5 * (X + np.swapaxes(X[neg], 1, 2))
    X[0] += 0.1 * np.eye(D)
    return X


# Benchmark workloads: (name, lattice spins per axis, cluster spins per axis, field h).
WORKLOADS = {
    # 1-D transverse-field Ising chain, h = 1, 2-spin clusters (16 x 16 pair marginals),
    # 4096 clusters = 4096 wavevectors (8192 spins)
    "tfim1d_L2_N4096": dict(lattice=(8192,), cluster=(2,), h=1.0, kind="tfim"),
    # the same chain at 4096 spins (2048 clusters)
    "tfim1d_L2_N2048": dict(lattice=(4096,), cluster=(2,), h=1.0, kind="tfim"),
    # the paper's table instance: TFI 100 x 1 periodic, h = 1, 2 x 1 clusters (50 clusters)
    "tfim1d_L2_N50": dict(lattice=(100,), cluster=(2,), h=1.0, kind="tfim"),
    # 1-D TFI chain, 16 spins, single-spin clusters (4 x 4 pair marginals)
    "tfim1d_L1_N16": dict(lattice=(16,), cluster=(1,), h=1.0, kind="tfim"),
    # 2-D square lattice 64 x 64, h = 3, 2 x 1 clusters (16 x 16 pair marginals), 32 x 64 clusters
    "tfim2d_L2_64x64": dict(lattice=(64, 64), cluster=(2, 1), h=3.0, kind="tfim"),
    # 1-D TFI chain of 4096 spins, h = 1, 4-spin clusters (16 x 16 cluster marginals, 256 x 256
    # pair marginals), 1024 clusters
    "tfim1d_L4_N1024": dict(lattice=(4096,), cluster=(4,), h=1.0, kind="tfim"),
    # 2-D square lattice 64 x 64, h = 3, 2 x 2 clusters (256 x 256 pair marginals), 32 x 32 clusters
    "tfim2d_L4_32x32": dict(lattice=(64, 64), cluster=(2, 2), h=3.0, kind="tfim"),
    # the 4-spin-cluster chain at 1024 spins (256 clusters): a D = 256 case small enough for
    # profiler captures (a few GB on the device)
    "tfim1d_L4_N256": dict(lattice=(1024,), cluster=(4,), h=1.0, kind="tfim"),
}


def _supported_clusters(n):
    """Nearest cluster count to n that the solver's block DFT supports for a 1-D chain: any n
    up to 64, else n = n1 * n2 with n1, n2 <= 64."""
    def ok(k):
        if 2 <= k <= 64:
            return True
        return 64 < k <= 4096 and any(k % a == 0 and k // a <= 64 for a in range(2, 65))
    for d in range(0, 4096):
        for k in (n - d, n + d):
            if ok(k):
                return k
    raise ValueError(n)


def batch_instances(family="c4", count=256, seed=None):
    """Independent 1-D instances: list of dict(kind, x, lattice, cluster).

    c4:    half TFI (h ~ U[0.2, 2.0]), half XXZ (Delta ~ U[0, 1.5]); chain length log-uniform in
           [64, 8192] spins; 2- or 3-spin clusters (16 x 16 or 64 x 64 pair marginals); the
           cluster count is rounded to one the block DFT supports.
    paper: TFI chains of 100 spins with 2-spin clusters (the paper's table instance), h ~ U[0.2, 2].
    """
    rng = _rng(seed)
    out = []
    for i in range(count):
        if family == "paper":
            out.append(dict(kind="tfim", x=float(rng.uniform(0.2, 2.0)), lattice=(100,), cluster=(2,)))
            continue
        kind = "tfim" if i < count // 2 else "xxz"
        x = float(rng.uniform(0.2, 2.0) if kind == "tfim" else rng.uniform(0.0, 1.5))
        L = int(rng.integers(2, 4))
        length = float(np.exp(rng.uniform(np.log(64), np.log(8192))))
        n = _supported_clusters(max(2, int(round(length / L))))
        out.append(dict(kind=kind, x=x, lattice=(n * L,), cluster=(L,)))
    return out


_PX = np.array([[0.0, 1.0], [1.0, 0.0]])
_PZ = np.array([[1.0, 0.0], [0.0, -1.0]])
_PYPY = np.array([[0.0, 0.0, 0.0, -1.0], [0.0, 0.0, 1.0, 0.0], [0.0, 1.0, 0.0, 0.0],
                  [-1.0, 0.0, 0.0, 0.0]])  # sigma^y (x) sigma^y, real


# General (not translation-invariant) workloads: (spins, spins per cluster, model, alpha).
GENERAL_WORKLOADS = {
    # disordered TFI chain of 128 spins with all-to-all 1/r^2 couplings, single-spin clusters:
    # 8128 pairs of 4 x 4 marginals, X of 512 x 512
    "lrtfim_N128_L1": dict(nspins=128, L=1, kind="tfim", alpha=2.0),
    # disordered XXZ chain of 64 spins, all-to-all 1/r^2, 2-spin clusters: 496 pairs of 16 x 16
    # marginals, X of 512 x 512
    "lrxxz_N64_L2": dict(nspins=64, L=2, kind="xxz", alpha=2.0),
    # the paper's fermionic benchmarks: spinless fermions on a 20-site ring, 2-site clusters
    # (45 pairs of 16 x 16 marginals, X of 160 x 160), short-range U = 2 and long-range U = 1
    "sf_N20_L2": dict(nsites=20, L=2, kind="fermion", U=2.0, long_range=False),
    "lrsf_N20_L2": dict(nsites=20, L=2, kind="fermion", U=1.0, long_range=True),
}


def general_terms(name):
    """(terms, sites per cluster) of a general workload: spin terms (dict with nspins) or
    spinless-fermion terms (dict with nsites)."""
    w = GENERAL_WORKLOADS[name]
    if w["kind"] == "fermion":
        return fermion_ring(w["nsites"], w["U"], long_range=w["long_range"]), w["L"]
    return disordered_chain(w["nspins"], w["kind"], alpha=w["alpha"]), w["L"]


def disordered_chain(nspins, kind="tfim", alpha=2.0, seed=None, field=(0.5, 1.5)):
    """An open chain of `nspins` spin-1/2 with random fields and all-to-all couplings decaying as
    1 / |s - t|^alpha, as terms: dict(onsite (nspins, 2, 2), bond_sites (nb, 2) int32 with s < t,
    bond_ops (nb, 4, 4), spin s the first factor).

    tfim: H = -sum_s h_s X_s - sum_{s<t} J_st Z_s Z_t,
    xxz:  H = sum_{s<t} J_st (X_s X_t + Y_s Y_t + Delta_s Z_s Z_t) - sum_s h_s Z_s / 10,
    with h_s ~ U[field], J_st = xi_st / |s - t|^alpha, xi_st ~ U[0.5, 1.5], Delta_s ~ U[0, 1.5]."""
    rng = _rng(seed)
    h = rng.uniform(field[0], field[1], size=nspins)
    sites = np.array([(s, t) for s in range(nspins) for t in range(s + 1, nspins)],
                     dtype=np.int32).reshape(-1, 2)
    xi = rng.uniform(0.5, 1.5, size=len(sites))
    J = xi / np.abs(sites[:, 1] - sites[:, 0]).astype(np.float64) ** alpha
    if kind == "tfim":
        onsite = -h[:, None, None] * _PX
        ops = -J[:, None, None] * np.kron(_PZ, _PZ)
    else:
        delta = rng.uniform(0.0, 1.5, size=nspins)
        onsite = -0.1 * h[:, None, None] * _PZ
        ops = J[:, None, None] * (np.kron(_PX, _PX) + _PYPY
                                  + delta[sites[:, 0], None, None] * np.kron(_PZ, _PZ))
    return dict(nspins=nspins, onsite=onsite, bond_sites=sites, bond_ops=ops)


def fermion_ring(nsites, U, long_range=False):
    """Spinless fermions on a periodic ring (the paper's fermionic examples): hopping -1 on each
    ring bond, and U (n_i - 1/2)(n_j - 1/2) on each bond, or, long-range, U / d(i, j) for every
    ordered pair i != j (2 U / d per unordered pair, d the distance on the ring).
    Returns dict(nsites, hops [(i, j, t)], pairs [(i, j, v)]) with i < j."""
    bonds = sorted({tuple(sorted((i, (i + 1) % nsites))) for i in range(nsites)})
    hops = [(i, j, -1.0) for i, j in bonds]
    if long_range:
        pairs = [(i, j, 2.0 * U / min(j - i, nsites - (j - i)))
                 for i in range(nsites) for j in range(i + 1, nsites)]
    else:
        pairs = [(i, j, float(U)) for i, j in bonds]
    return dict(nsites=nsites, hops=hops, pairs=pairs)
