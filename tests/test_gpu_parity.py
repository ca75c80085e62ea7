"""GPU parity: every step of the sweep through the C ABI against the CPU oracle, element by
element, on the same seeded inputs.

Tolerances (float64 mode): 1e-10 relative to the largest entry of the compared array (states)
or to the value itself (energy, residual, bound), the target for float64 results at every D;
both sides run the same float64 arithmetic in a different order (Jacobi vs LAPACK eigensolver,
FFT vs numpy FFT), so agreement is ~1e-13 in practice.  Float32
projections (VE_PREC_MIXED) are held to 8 (n + 16) 2^-24 ||A||_2 per entry: a float32 Jacobi
eigensolve of an n x n matrix runs ~10 sweeps of n - 1 rounds, and the measured error is
(20 + 1.3 n) 2^-24 ||A||_2 at n = 4 .. 64, so this keeps a ~4x margin.  The final certified
bound of a mixed solve is held to 1e-6 per spin.  Double-float results (VE_PREC_DF64) are held
to the float64 tolerances times 2^(53-48) = 32, the ratio of the two unit roundoffs; after 30
sweeps the measured state error is 5-13x that of float64 mode (at most 6.2e-10, D = 256).
"""
import os

import numpy as np
import pytest

import __graft_entry__
from oracle import models as mo
from oracle import ve_oracle as vo
from paper_2106_02682_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL64 = 1e-10
RTOL32 = 2e-5    # relative tolerance of float32 results on O(1) arrays (X step, 16 x 16 blocks)
# Double-float words carry a 48-bit significand (unit roundoff ~2^-48 against float64's 2^-53):
# the float64 tolerance scaled by that ratio.
RTOL_DF64 = RTOL64 * 2.0 ** (53 - 48)


def state_tol(prec):
    """Relative tolerance of whole-state comparisons for precision mode 0 (float64) or 2 (df64)."""
    return RTOL64 if prec == 0 else RTOL_DF64


def close(a, b, prec):
    """Scalar results (energy, residual, bound terms): relative to the value, absolute below 1."""
    return abs(a - b) <= state_tol(prec) * max(1.0, abs(b))


def tol32(A):
    """Per-entry tolerance of a float32 projection of the n x n matrix A."""
    return 8.0 * (A.shape[-1] + 16) * 2.0 ** -24 * np.linalg.norm(A, 2)


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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# ------------------------------------------------------------------ S3: pair projections

@pytest.mark.parametrize("n", [2, 4, 8, 16, 64])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_project_sym_matches_oracle(ve, n, prec):
    A = synth.symmetric_batch(1001 if n <= 16 else 131, n, seed=n)
    x = dev(A)
    y = torch.empty_like(x)
    ve.ve_project_psd_sym(x.data_ptr(), y.data_ptr(), n, A.shape[0], prec)
    torch.cuda.synchronize()
    ref = vo.proj_psd(A)
    out = y.cpu().numpy()
    for b in range(A.shape[0]):
        tol = state_tol(prec) * max(1.0, np.max(np.abs(A[b]))) if prec != 1 else tol32(A[b])
        assert np.max(np.abs(out[b] - ref[b])) <= tol, b
    # in place, and an empty batch
    ve.ve_project_psd_sym(x.data_ptr(), x.data_ptr(), n, A.shape[0], prec)
    ve.ve_project_psd_sym(x.data_ptr(), x.data_ptr(), n, 0, prec)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy(), out)


@pytest.mark.parametrize("n", [4, 16, 64])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_project_herm_matches_oracle(ve, n, prec):
    A = synth.hermitian_batch(517 if n <= 16 else 67, n, seed=100 + n)
    inter = np.stack([A.real, A.imag], axis=-1)
    x = dev(inter)
    y = torch.empty_like(x)
    ve.ve_project_psd_herm(x.data_ptr(), y.data_ptr(), n, A.shape[0], prec)
    torch.cuda.synchronize()
    o = y.cpu().numpy()
    out = o[..., 0] + 1j * o[..., 1]
    ref = vo.proj_psd(A)
    for b in range(A.shape[0]):
        tol = state_tol(prec) * max(1.0, np.max(np.abs(A[b]))) if prec != 1 else tol32(A[b])
        assert np.max(np.abs(out[b] - ref[b])) <= tol, b


def test_projection_degenerate_cases(ve):
    n = 16
    cases = [np.zeros((n, n)), np.eye(n), -np.eye(n), np.diag(np.r_[np.ones(8), -np.ones(8)]),
             np.ones((n, n)), -np.ones((n, n)), 1e-300 * np.eye(n), 1e12 * synth.symmetric_batch(1, n, 5)[0]]
    A = np.array(cases)
    x = dev(A)
    y = torch.empty_like(x)
    ve.ve_project_psd_sym(x.data_ptr(), y.data_ptr(), n, len(cases), 0)
    torch.cuda.synchronize()
    out = y.cpu().numpy()
    ref = vo.proj_psd(A)
    for b in range(len(cases)):
        assert np.max(np.abs(out[b] - ref[b])) <= RTOL64 * max(1.0, np.max(np.abs(A[b]))), b


@pytest.mark.parametrize("n,herm", [(256, False), (512, False), (256, True)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_large_projection_matches_oracle(ve, n, herm, prec):
    """n = 256, 512 staged in a caller workspace (the 4-spin-cluster blocks, and the kernel-only
    512 x 512 batch); the first matrix of each batch has eigenvalues +1, -1, 0 repeated."""
    count = 3 if n == 256 else 2
    A = (synth.hermitian_batch(count, n, seed=n + 11) if herm
         else synth.symmetric_batch(count, n, seed=n + 5))
    host = np.stack([A.real, A.imag], axis=-1) if herm else A
    x = dev(host)
    y = torch.empty_like(x)
    ws_bytes = ve.ve_project_psd_large_workspace_size(n, herm, prec)
    assert ws_bytes > 0
    ws = torch.empty(ws_bytes // 8 + 1, dtype=torch.float64, device="cuda")
    fn = ve.ve_project_psd_herm_large if herm else ve.ve_project_psd_sym_large
    fn(x.data_ptr(), y.data_ptr(), n, count, ws.data_ptr(), ws_bytes, prec)
    torch.cuda.synchronize()
    o = y.cpu().numpy()
    out = o[..., 0] + 1j * o[..., 1] if herm else o
    ref = vo.proj_psd(A)
    for b in range(count):
        if prec == 1:
            tol = tol32(A[b])
        else:
            tol = state_tol(prec) * max(1.0, np.max(np.abs(A[b])))
        assert np.max(np.abs(out[b] - ref[b])) <= tol, (b, np.max(np.abs(out[b] - ref[b])), tol)
    # in place, an empty batch, and a workspace one byte short
    fn(x.data_ptr(), x.data_ptr(), n, count, ws.data_ptr(), ws_bytes, prec)
    fn(x.data_ptr(), x.data_ptr(), n, 0, ws.data_ptr(), ws_bytes, prec)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy(), o)
    with pytest.raises(ve.VEError):
        fn(x.data_ptr(), y.data_ptr(), n, count, ws.data_ptr(), ws_bytes - 1, prec)


# ------------------------------------------------------------------ S7-S9: the X step

CIRC = [((2,), 4), ((3,), 16), ((5,), 4), ((6,), 16), ((16,), 16), ((50,), 16), ((64,), 16),
        ((100,), 4), ((96,), 16),
        ((2048,), 16), ((4096,), 4), ((2, 3), 16), ((4, 4), 4), ((8, 6), 16), ((32, 32), 16),
        ((3,), 64), ((2, 2), 64)]


@pytest.mark.parametrize("M,D", CIRC)
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_circulant_projection_matches_oracle(ve, M, D, prec):
    if prec != 0 and D == 4 and np.prod(M) > 1000:
        pytest.skip("covered by the float64 case")
    X = synth.circulant_first_row(M, D, seed=int(np.prod(M)) + D)
    ref = np.real(vo._lattice_dft(vo.proj_psd(vo._lattice_dft(X, M, False)), M, True))
    ws_bytes = ve.ve_circulant_workspace_size(M, D)
    ws = torch.empty(ws_bytes // 8 + 64, dtype=torch.float64, device="cuda")
    x = dev(X)
    y = torch.empty_like(x)
    ve.ve_circulant_project(x.data_ptr(), y.data_ptr(), M, D, ws.data_ptr(), ws_bytes, prec)
    torch.cuda.synchronize()
    err = relerr(y.cpu().numpy(), ref)
    assert err <= (10 * RTOL32 if prec == 1 else state_tol(prec)), err
    # in place
    ve.ve_circulant_project(x.data_ptr(), x.data_ptr(), M, D, ws.data_ptr(), ws_bytes, prec)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_circulant_projection_rejects_small_workspace(ve):
    M, D = (16,), 16
    ws_bytes = ve.ve_circulant_workspace_size(M, D)
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device="cuda")
    x = torch.zeros(16 * D * D, dtype=torch.float64, device="cuda")
    with pytest.raises(ve.VEError):
        ve.ve_circulant_project(x.data_ptr(), x.data_ptr(), M, D, ws.data_ptr(), ws_bytes - 256, 0)


# ------------------------------------------------------------------ whole sweeps

SWEEP_CASES = [
    ((16,), (1,), "tfim", 1.0),
    ((8,), (2,), "tfim", 0.7),
    ((3,), (1,), "xxz", 0.4),
    ((100,), (1,), "tfim", 0.5),
    ((192,), (2,), "tfim", 1.2),
    ((4, 4), (1, 1), "tfim", 2.0),
    ((4, 6), (2, 1), "xxz", 0.5),
    ((6, 4), (1, 2), "tfim", 3.0),
    ((12,), (3,), "tfim", 1.0),
    ((6, 4), (3, 1), "xxz", 1.0),
    ((8,), (4,), "tfim", 1.0),
    ((16,), (4,), "xxz", 0.7),
    ((4, 4), (2, 2), "tfim", 3.0),
]


def _terms(kind, dim, x):
    return mo.tfim_terms(1.0, x, dim) if kind == "tfim" else mo.xxz_terms(1.0, x, dim)


def _ham(ve, kind, dim, x):
    return ve.ve_ham_tfim(dim, 1.0, x) if kind == "tfim" else ve.ve_ham_xxz(dim, 1.0, x)


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("lattice,cluster,kind,x", SWEEP_CASES)
def test_sweeps_match_oracle(ve, lattice, cluster, kind, x, prec):
    """float64 (prec 0) and double-float (prec 2) sweeps against the oracle."""
    dim = len(lattice)
    pb = vo.Problem(mo.cluster_model(lattice, cluster, *_terms(kind, dim, x)))
    st = vo.initial_state(pb)
    h = ve.ve_create(lattice, cluster, _ham(ve, kind, dim, x), ve.ve_default_options(precision=prec))
    try:
        assert ve.ve_dims(h) == (pb.N, pb.m, pb.D)
        np.testing.assert_array_equal(ve.ve_get_state(h), vo.pack_state(pb, st))
        done = 0
        for k in (1, 6, 23):
            code, status = ve.ve_iterate(h, k, 0.0)
            for _ in range(k):
                diag = vo.iterate(pb, st)
            done += k
            assert code == 0 and status.iter == done
            err = relerr(ve.ve_get_state(h), vo.pack_state(pb, st))
            assert err < state_tol(prec), (done, err)
            assert close(status.energy_per_spin, diag['energy'], prec)
            assert close(status.feas_err, diag['feas_err'], prec)
            if done > 1:
                assert close(status.d_energy, diag['d_energy'], prec)
        cert = ve.ve_bound(h)
        ocert = vo.certified_bound(pb, st)
        for key in ('bound_per_spin', 'raw_bound', 'x_neg_correction', 'primal_per_spin'):
            assert close(getattr(cert, key), ocert[key], prec), key
        assert abs(cert.x_min_eig - ocert['x_min_eig']) < 1e-9
    finally:
        ve.ve_destroy(h)


@pytest.mark.parametrize("prec", [0, 2])
def test_full_size_workload_matches_oracle(ve, prec):
    """The benchmark workload (1-D TFI, h = 1, 2-spin clusters, 4096 clusters = 4096
    wavevectors, D = 16), three sweeps, compared over the whole state."""
    lattice, cluster = (8192,), (2,)
    pb = vo.Problem(mo.cluster_model(lattice, cluster, *mo.tfim_terms(1.0, 1.0, 1)))
    st = vo.initial_state(pb)
    h = ve.ve_create(lattice, cluster, ve.ve_ham_tfim(1, 1.0, 1.0), ve.ve_default_options(precision=prec))
    try:
        _, status = ve.ve_iterate(h, 3, 0.0)
        for _ in range(3):
            diag = vo.iterate(pb, st)
        tol = state_tol(prec)
        assert relerr(ve.ve_get_state(h), vo.pack_state(pb, st)) < tol
        assert abs(status.energy_per_spin - diag['energy']) < tol
        cert = ve.ve_bound(h)
        assert abs(cert.bound_per_spin - vo.certified_bound(pb, st)['bound_per_spin']) < tol
    finally:
        ve.ve_destroy(h)


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("lattice,cluster,kind,x,sweeps", [((100,), (2,), "tfim", 1.0, 300),
                                                          ((16,), (4,), "xxz", 0.7, 80)])
def test_first_order_stop_matches_oracle(ve, lattice, cluster, kind, x, sweeps, prec):
    """Long runs in which the warm-started eigensolves end mostly with the first-order
    (Daleckii-Krein) reconstruction -- the branch every steady-state sweep takes -- against the
    oracle's exact eigendecompositions: the branch must have fired in both the pair and the
    wavevector projections, and the whole state, the status and the certificate must still agree
    to the float64 (double-float) tolerance.  The paper's 100-spin table instance (D = 16) and a
    4-spin-cluster chain (D = 256)."""
    dim = len(lattice)
    pb = vo.Problem(mo.cluster_model(lattice, cluster, *_terms(kind, dim, x)))
    st = vo.initial_state(pb)
    for _ in range(sweeps):
        diag = vo.iterate(pb, st)
    h = ve.ve_create(lattice, cluster, _ham(ve, kind, dim, x), ve.ve_default_options(precision=prec))
    try:
        ve.ve_iterate(h, 1, 0.0)
        ve.ve_profile(h, 1)
        _, status = ve.ve_iterate(h, sweeps - 1, 0.0)
        (fo_pair, n_pair), (fo_k, n_k) = ve.ve_profile_first_order(h)
        ve.ve_profile(h, 0)
        assert n_pair > 0 and n_k > 0
        assert fo_pair >= n_pair // 4 and fo_k >= n_k // 4, (fo_pair, n_pair, fo_k, n_k)
        err = relerr(ve.ve_get_state(h), vo.pack_state(pb, st))
        assert err < state_tol(prec), err
        assert close(status.energy_per_spin, diag['energy'], prec)
        assert close(status.feas_err, diag['feas_err'], prec)
        cert = ve.ve_bound(h)
        ocert = vo.certified_bound(pb, st)
        for key in ('bound_per_spin', 'raw_bound', 'primal_per_spin'):
            assert close(getattr(cert, key), ocert[key], prec), key
    finally:
        ve.ve_destroy(h)


def _swap_image(B, m):
    """P B P for D x D blocks (last two axes), P exchanging the two clusters' factors."""
    sw = np.array([b * m + a for a in range(m) for b in range(m)])
    return B[..., sw, :][..., :, sw]


@pytest.mark.parametrize("lattice,cluster,kind,x", [((12,), (2,), "tfim", 0.8),
                                                   ((4, 6), (2, 1), "xxz", 0.5),
                                                   ((8,), (4,), "tfim", 1.0)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_tied_offsets_are_swap_images(ve, lattice, cluster, kind, x, prec):
    """After sweeps from the initial state the -delta blocks are the swap images of the delta
    blocks: rho~ and Lambda conjugated by the factor exchange and Lambda1, Lambda2 exchanged,
    bit for bit; X_{0,-delta} = X_{0,delta}^T to the rounding of the DFT."""
    dim = len(lattice)
    pb = vo.Problem(mo.cluster_model(lattice, cluster, *_terms(kind, dim, x)))
    h = ve.ve_create(lattice, cluster, _ham(ve, kind, dim, x), ve.ve_default_options(precision=prec))
    try:
        ve.ve_iterate(h, 7, 0.0)
        st = vo.unpack_state(pb, ve.ve_get_state(h))
    finally:
        ve.ve_destroy(h)
    neg = vo.neg_index(pb.M)
    tied = neg[1:] != np.arange(1, pb.N)  # offsets with -delta != delta; the others are
    img = neg[1:][tied] - 1               # updated on their own, symmetric to rounding
    for key in ('rt', 'lam'):
        np.testing.assert_array_equal(st[key][img], _swap_image(st[key], pb.m)[tied])
        assert relerr(st[key][~tied], _swap_image(st[key], pb.m)[~tied]) < (
            10 * RTOL32 if prec == 1 else state_tol(prec))
    np.testing.assert_array_equal(st['lam1'][img], st['lam2'][tied])
    np.testing.assert_array_equal(st['lam2'][img], st['lam1'][tied])
    xerr = relerr(st['X'][neg], np.swapaxes(st['X'], 1, 2))
    assert xerr < (10 * RTOL32 if prec == 1 else state_tol(prec)), xerr


def test_first_sweep_takes_the_canonical_members(ve):
    """A state set without the swap symmetry between delta and -delta: a sweep reads, of each
    pair {delta, -delta}, the member with the smaller linear index, so it matches the oracle's
    sweep from the state whose other members are replaced by the images of those."""
    lattice, cluster = (12,), (2,)
    pb = vo.Problem(mo.cluster_model(lattice, cluster, *mo.tfim_terms(1.0, 0.8, 1)))
    st = vo.initial_state(pb)
    for _ in range(4):
        vo.iterate(pb, st)
    g = np.random.default_rng(7)
    symn = lambda *shape: (lambda Z: 0.5 * (Z + np.swapaxes(Z, -1, -2)))(g.normal(size=shape))
    P, D, m = pb.N - 1, pb.D, pb.m
    st['rt'] = st['rt'] + 1e-3 * symn(P, D, D)
    st['lam'] = st['lam'] + 1e-3 * symn(P, D, D)
    st['lam1'] = st['lam1'] + 1e-3 * symn(P, m, m)
    st['lam2'] = st['lam2'] + 1e-3 * symn(P, m, m)
    st['X'] = st['X'] + 1e-3 * g.normal(size=st['X'].shape)
    neg = vo.neg_index(pb.M)
    for dl in range(pb.N):
        if neg[dl] == dl:  # offsets with -delta = delta (and X_00) keep the swap symmetry
            st['X'][dl] = 0.5 * (st['X'][dl] + st['X'][dl].T)
            if dl > 0:
                for key in ('rt', 'lam'):
                    st[key][dl - 1] = 0.5 * (st[key][dl - 1] + _swap_image(st[key][dl - 1], m))
                l12 = 0.5 * (st['lam1'][dl - 1] + st['lam2'][dl - 1])
                st['lam1'][dl - 1], st['lam2'][dl - 1] = l12, l12.copy()
    given = vo.pack_state(pb, st)
    for dl in range(1, pb.N):
        nd = neg[dl]
        if nd < dl:
            st['rt'][dl - 1] = _swap_image(st['rt'][nd - 1], m)
            st['lam'][dl - 1] = _swap_image(st['lam'][nd - 1], m)
            st['lam1'][dl - 1] = st['lam2'][nd - 1]
            st['lam2'][dl - 1] = st['lam1'][nd - 1]
            st['X'][dl] = st['X'][nd].T
    assert relerr(given, vo.pack_state(pb, st)) > 1e-4  # the given state lacks the symmetry
    h = ve.ve_create(lattice, cluster, ve.ve_ham_tfim(1, 1.0, 0.8))
    try:
        ve.ve_set_state(h, given)
        ve.ve_iterate(h, 1, 0.0)
        vo.iterate(pb, st)
        assert relerr(ve.ve_get_state(h), vo.pack_state(pb, st)) < RTOL64
    finally:
        ve.ve_destroy(h)


def test_state_roundtrip_resume_and_determinism(ve):
    """Two handles with the same history agree bitwise.  A state read and set back on the same
    handle continues bit for bit (the handle keeps the eigenvectors of its last projections as
    the eigensolves' starting point); on a fresh handle the eigensolves restart cold, so the run
    matches an uninterrupted one to rounding."""
    lattice, cluster = (64,), (2,)
    ham = ve.ve_ham_tfim(1, 1.0, 0.9)
    a, b, c, d = (ve.ve_create(lattice, cluster, ham), ve.ve_create(lattice, cluster, ham),
                  ve.ve_create(lattice, cluster, ham), ve.ve_create(lattice, cluster, ham))
    try:
        ve.ve_iterate(a, 40, 0.0)
        ve.ve_iterate(c, 40, 0.0)
        np.testing.assert_array_equal(ve.ve_get_state(a), ve.ve_get_state(c))
        ve.ve_iterate(b, 25, 0.0)
        snap = ve.ve_get_state(b)
        ve.ve_set_state(b, snap)
        ve.ve_iterate(b, 15, 0.0)
        np.testing.assert_array_equal(ve.ve_get_state(b), ve.ve_get_state(a))
        ve.ve_set_state(d, snap)
        ve.ve_iterate(d, 15, 0.0)
        assert relerr(ve.ve_get_state(d), ve.ve_get_state(a)) < 1e-12
        with pytest.raises(ve.VEError):
            ve.ve_set_state(b, snap[:-1])
        st = ve.ve_get_status(b)
        assert st.iter == 40
    finally:
        for x in (a, b, c, d):
            ve.ve_destroy(x)


def test_dft_tuning_is_cached_and_changes_no_result(ve, tmp_path, monkeypatch):
    """The first sweep times the DFT passes' launch shapes once per shape and precision; the
    choice goes to the VE_TUNE_CACHE file, is reused by a second handle, and the sweeps still
    match the oracle."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("VE_TUNE_CACHE", str(path))
    lattice, cluster = (2 * 91,), (2,)  # 91 clusters: a shape no other test uses
    pb = vo.Problem(mo.cluster_model(lattice, cluster, *mo.tfim_terms(1.0, 0.9, 1)))
    st = vo.initial_state(pb)
    h1 = ve.ve_create(lattice, cluster, ve.ve_ham_tfim(1, 1.0, 0.9))
    h2 = ve.ve_create(lattice, cluster, ve.ve_ham_tfim(1, 1.0, 0.9))
    try:
        ve.ve_iterate(h1, 5, 0.0)
        lines = path.read_text().splitlines()
        assert len(lines) == 1 and "M91x1_D16_f64" in lines[0], lines
        ve.ve_iterate(h2, 5, 0.0)
        assert path.read_text().splitlines() == lines
        np.testing.assert_array_equal(ve.ve_get_state(h1), ve.ve_get_state(h2))
        for _ in range(5):
            vo.iterate(pb, st)
        assert relerr(ve.ve_get_state(h1), vo.pack_state(pb, st)) < RTOL64
    finally:
        ve.ve_destroy(h1)
        ve.ve_destroy(h2)


def test_nonfinite_state_is_reported(ve):
    h = ve.ve_create((16,), (1,), ve.ve_ham_tfim(1, 1.0, 1.0))
    try:
        s = ve.ve_get_state(h)
        s[0] = np.nan
        ve.ve_set_state(h, s)
        code = ve.lib.ve_iterate(ve.c_void_p(h), 10, 0.0, None)
        assert code == ve.VE_ENONFINITE
    finally:
        ve.ve_destroy(h)


def test_tensor_core_waits_time_out_cleanly(ve):
    """Failure detection without a GPU fault: a tensor-core product whose loads are withheld must
    see its bounded waits run out, report the timeout and return within a few seconds (not
    hang), and the same context must then run the product cleanly."""
    sec = ve.ve_selftest_bounded_wait()
    assert 0.5 < sec < 10.0, sec


def test_converges_to_the_paper_table_value(ve):
    """TFI 20x1, 2x1 clusters, h = 1 (Sec. 4 table): 10 000 sweeps on the GPU."""
    h = ve.ve_create((20,), (2,), ve.ve_ham_tfim(1, 1.0, 1.0))
    try:
        _, st = ve.ve_iterate(h, 10000, 0.0)
        cert = ve.ve_bound(h)
        assert abs(st.energy_per_spin - (-1.283534)) < 5e-6
        assert -1.283534 - 5e-6 < cert.bound_per_spin <= -1.283534 + 1e-7
    finally:
        ve.ve_destroy(h)


def test_mixed_precision_reaches_the_float64_bound(ve):
    """Float64, mixed-precision and double-float solves of the same instance, each run to
    30 000 sweeps with a 1e-9 target: their certified bounds agree within 1e-6 per spin and lie
    below the exact (Jordan-Wigner) energy."""
    lattice, cluster = (32,), (2,)
    ham = ve.ve_ham_tfim(1, 1.0, 1.0)
    out = {}
    for prec in (0, 1, 2):
        h = ve.ve_create(lattice, cluster, ham, ve.ve_default_options(precision=prec))
        try:
            ve.ve_iterate(h, 30000, 1e-9)
            out[prec] = ve.ve_bound(h).bound_per_spin
        finally:
            ve.ve_destroy(h)
    assert abs(out[0] - out[1]) < 1e-6 and abs(out[0] - out[2]) < 1e-6, out
    assert max(out.values()) <= mo.tfim_chain_jw_energy(32, 1.0, 1.0) / 32


@pytest.mark.parametrize("lattice,cluster", [((64,), (2,)), ((16,), (4,)), ((4, 6), (2, 2))])
def test_mixed_sweeps_track_the_oracle(ve, lattice, cluster):
    """Mixed-precision sweeps (float32 arithmetic in the pair pass, the DFT and both
    projections; float64 state and reductions) stay within float32 rounding of the float64
    oracle: the whole state after 30 sweeps within 30 times the per-sweep bound of a float32
    projection, 8 (D + 16) 2^-24, relative (the sweep is nonexpansive, so errors add at most
    linearly): 4.6e-4 at D = 16, 3.9e-3 at D = 256.  At D = 256 (a chain of 4-spin clusters and
    a 2-D lattice of 2 x 2 clusters) the projections run on the tensor cores with block Jacobi."""
    dim = len(lattice)
    pb = vo.Problem(mo.cluster_model(lattice, cluster, *mo.tfim_terms(1.0, 0.8, dim)))
    st = vo.initial_state(pb)
    h = ve.ve_create(lattice, cluster, ve.ve_ham_tfim(dim, 1.0, 0.8),
                     ve.ve_default_options(precision=1))
    try:
        ve.ve_iterate(h, 30, 0.0)
        for _ in range(30):
            vo.iterate(pb, st)
        err = relerr(ve.ve_get_state(h), vo.pack_state(pb, st))
        assert err < 30 * 8 * (pb.D + 16) * 2.0 ** -24, err
        cert = ve.ve_bound(h)
        assert abs(cert.bound_per_spin - vo.certified_bound(pb, st)['bound_per_spin']) < 1e-3
    finally:
        ve.ve_destroy(h)


@pytest.mark.parametrize("lattice,cluster,x", [((4096,), (4,), 1.0), ((64, 64), (2, 2), 3.0)])
def test_full_size_4spin_chain_mixed_matches_oracle(ve, lattice, cluster, x):
    """The two 4-spin-cluster benchmark workloads themselves -- the 4096-spin chain and the 2-D
    64 x 64 lattice in 2 x 2 clusters (1024 clusters each, D = 256: 513 / 514 canonical wavevector
    blocks and 512 pair blocks per projection batch) -- in mixed precision, the tensor-core path
    as the benchmark runs it (captured sweep graph after the first sweep), two sweeps from the
    cold start against the float64 oracle over the whole state: within twice the per-sweep
    float32 bound of the test above, and the certificate within 1e-3 per spin."""
    dim = len(lattice)
    vo.set_threads(os.cpu_count() or 1)
    try:
        pb = vo.Problem(mo.cluster_model(lattice, cluster, *mo.tfim_terms(1.0, x, dim)))
        st = vo.initial_state(pb)
        h = ve.ve_create(lattice, cluster, ve.ve_ham_tfim(dim, 1.0, x),
                         ve.ve_default_options(precision=1))
        try:
            ve.ve_iterate(h, 2, 0.0)
            for _ in range(2):
                vo.iterate(pb, st)
            err = relerr(ve.ve_get_state(h), vo.pack_state(pb, st))
            assert err < 2 * 8 * (pb.D + 16) * 2.0 ** -24, err
            cert = ve.ve_bound(h)
            assert abs(cert.bound_per_spin - vo.certified_bound(pb, st)['bound_per_spin']) < 1e-3
        finally:
            ve.ve_destroy(h)
    finally:
        vo.set_threads(1)


# ------------------------------------------------------------------ batches of instances

BATCH = [((100,), (2,), "tfim", 1.0), ((16,), (1,), "tfim", 0.5), ((24,), (2,), "xxz", 0.8),
         ((4, 4), (1, 1), "tfim", 2.0), ((12,), (3,), "xxz", 1.0), ((96,), (2,), "tfim", 1.5)]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_reproduces_single_handles(ve, prec):
    """A batch advances every instance exactly as a single handle would: same states bit for
    bit after a fixed number of sweeps and, with a tolerance, the same stopping sweep."""
    opt = ve.ve_default_options(precision=prec)
    inst = [(lat, clu, _ham(ve, kind, len(lat), x)) for lat, clu, kind, x in BATCH]
    for max_iter, tol in ((40, 0.0), (3000, 1e-4)):
        b = ve.ve_create_batch(inst, opt)
        try:
            code, sts = ve.ve_batch_iterate(b, max_iter, tol)
            states = [ve.ve_get_state(ve.ve_batch_handle(b, i)) for i in range(len(inst))]
            certs = ve.ve_batch_bound(b)
        finally:
            ve.ve_batch_destroy(b)
        for i, (lat, clu, hm) in enumerate(inst):
            h = ve.ve_create(lat, clu, hm, opt)
            try:
                c1, s1 = ve.ve_iterate(h, max_iter, tol)
                np.testing.assert_array_equal(states[i], ve.ve_get_state(h))
                assert s1.iter == sts[i].iter and s1.residual == sts[i].residual
                assert ve.ve_bound(h).bound_per_spin == certs[i].bound_per_spin
            finally:
                ve.ve_destroy(h)
