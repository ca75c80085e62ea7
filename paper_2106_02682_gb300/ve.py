"""ctypes binding of the C ABI in include/ve.h (argument marshalling only).

Every function keeps its C name.  Status codes < 0 raise VEError; VE_OK / VE_NOT_CONVERGED are
returned.  Device pointers are plain integers (e.g. torch_tensor.data_ptr()); streams are
integers (torch.cuda.Stream.cuda_stream) or None.  The shared library must have been built
(paper_2106_02682_gb300.build.build()); importing this module without it raises ImportError,
there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libve_gb300.so")

VE_OK = 0
VE_NOT_CONVERGED = 1
VE_EINVAL = -1
VE_ENOMEM = -2
VE_ECUDA = -3
VE_ENONFINITE = -4
VE_EUNSUPPORTED = -5
VE_ETIMEOUT = -6
VE_PREC_FP64 = 0
VE_PREC_MIXED = 1
VE_PREC_DF64 = 2
VE_MAX_BONDS = 4
VE_NSTAGE = 7
VE_NOALLOC_SCRATCH_BYTES = (16 << 20) + (256 << 10)
STAGES = ("pair", "rho0", "dual12", "status", "fft_forward", "xproj", "fft_inverse")
VE_GENERAL_NSTAGE = 4
GENERAL_STAGES = ("pair", "cluster", "dense_eig", "reconstruct")

c_int, c_long, c_double, c_void_p, c_size_t = (ctypes.c_int, ctypes.c_long, ctypes.c_double,
                                               ctypes.c_void_p, ctypes.c_size_t)
P_double = ctypes.POINTER(c_double)
P_float = ctypes.POINTER(ctypes.c_float)


class ve_lattice(ctypes.Structure):
    _fields_ = [("dim", c_int), ("extent", c_int * 2)]


class ve_cluster(ctypes.Structure):
    _fields_ = [("extent", c_int * 2)]


class ve_hamiltonian(ctypes.Structure):
    _fields_ = [("onsite", c_double * 4), ("nbond", c_int),
                ("bond_offset", (c_int * 2) * VE_MAX_BONDS),
                ("bond", (c_double * 16) * VE_MAX_BONDS)]


class ve_options(ctypes.Structure):
    _fields_ = [("mu", c_double), ("nu", c_double), ("eps", c_double), ("precision", c_int),
                ("check_every", c_int), ("stream", c_void_p)]


class ve_status(ctypes.Structure):
    _fields_ = [("iter", c_long), ("energy_per_spin", c_double), ("feas_err", c_double),
                ("d_energy", c_double), ("residual", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ve_cert(ctypes.Structure):
    _fields_ = [("bound_per_spin", c_double), ("raw_bound", c_double), ("x_min_eig", c_double),
                ("x_neg_correction", c_double), ("primal_per_spin", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ve_terms(ctypes.Structure):
    _fields_ = [("nspins", c_int), ("onsite", c_void_p), ("nbond", c_int),
                ("bond_sites", c_void_p), ("bond_ops", c_void_p)]


class ve_fermion_terms(ctypes.Structure):
    _fields_ = [("nsites", c_int), ("nhop", c_int), ("hop_sites", c_void_p), ("hop_t", c_void_p),
                ("npair", c_int), ("pair_sites", c_void_p), ("pair_v", c_void_p)]


class VEError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {ve_error_string(code)} ({code})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2106_02682_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    H = c_void_p
    sig = {
        "ve_default_options": (None, [ctypes.POINTER(ve_options)]),
        "ve_ham_tfim": (c_int, [c_int, c_double, c_double, ctypes.POINTER(ve_hamiltonian)]),
        "ve_ham_xxz": (c_int, [c_int, c_double, c_double, ctypes.POINTER(ve_hamiltonian)]),
        "ve_create": (c_int, [ctypes.POINTER(ve_lattice), ctypes.POINTER(ve_cluster),
                              ctypes.POINTER(ve_hamiltonian), ctypes.POINTER(ve_options),
                              ctypes.POINTER(H)]),
        "ve_iterate": (c_int, [H, c_long, c_double, ctypes.POINTER(ve_status)]),
        "ve_bound": (c_int, [H, ctypes.POINTER(ve_cert)]),
        "ve_destroy": (None, [H]),
        "ve_dims": (c_int, [H, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
        "ve_state_size": (c_size_t, [H]),
        "ve_get_state": (c_int, [H, P_double, c_size_t]),
        "ve_set_state": (c_int, [H, P_double, c_size_t]),
        "ve_get_status": (c_int, [H, ctypes.POINTER(ve_status)]),
        "ve_error_string": (ctypes.c_char_p, [c_int]),
        "ve_profile": (c_int, [H, c_int]),
        "ve_profile_read": (c_int, [H, P_double, ctypes.POINTER(c_long)]),
        "ve_profile_sweeps": (c_int, [H, P_double, P_double]),
        "ve_profile_first_order": (c_int, [H, ctypes.POINTER(c_long), ctypes.POINTER(c_long)]),
        "ve_selftest_bounded_wait": (c_int, [P_double]),
        "ve_create_batch": (c_int, [c_int, ctypes.POINTER(ve_lattice), ctypes.POINTER(ve_cluster),
                                    ctypes.POINTER(ve_hamiltonian), ctypes.POINTER(ve_options),
                                    ctypes.POINTER(c_void_p)]),
        "ve_batch_size": (c_int, [c_void_p]),
        "ve_batch_handle": (c_void_p, [c_void_p, c_int]),
        "ve_batch_iterate": (c_int, [c_void_p, c_long, c_double, ctypes.POINTER(ve_status)]),
        "ve_batch_bound": (c_int, [c_void_p, ctypes.POINTER(ve_cert)]),
        "ve_batch_destroy": (None, [c_void_p]),
        "ve_project_state_x": (c_int, [H]),
        "ve_mlp_create": (c_int, [c_int, c_int, c_int, c_int, ctypes.c_ulonglong,
                                  ctypes.POINTER(c_void_p)]),
        "ve_mlp_destroy": (None, [c_void_p]),
        "ve_mlp_num_params": (c_size_t, [c_void_p]),
        "ve_mlp_get_params": (c_int, [c_void_p, P_float, c_size_t]),
        "ve_mlp_set_params": (c_int, [c_void_p, P_float, c_size_t]),
        "ve_mlp_loss_grad": (c_int, [c_void_p, P_float, P_float, c_int, P_float, P_float]),
        "ve_mlp_train": (c_int, [c_void_p, P_float, P_float, c_int, c_int, ctypes.c_float, P_float]),
        "ve_mlp_predict": (c_int, [c_void_p, P_float, c_int, P_float]),
        "ve_project_psd_sym": (c_int, [c_void_p, c_void_p, c_int, c_long, c_int, c_void_p]),
        "ve_project_psd_herm": (c_int, [c_void_p, c_void_p, c_int, c_long, c_int, c_void_p]),
        "ve_project_psd_large_workspace_size": (c_size_t, [c_int, c_int, c_int]),
        "ve_project_psd_sym_large": (c_int, [c_void_p, c_void_p, c_int, c_long, c_int, c_void_p,
                                             c_size_t, c_void_p]),
        "ve_project_psd_herm_large": (c_int, [c_void_p, c_void_p, c_int, c_long, c_int, c_void_p,
                                              c_size_t, c_void_p]),
        "ve_circulant_workspace_size": (c_size_t, [c_int, ctypes.POINTER(c_int), c_int]),
        "ve_circulant_project": (c_int, [c_void_p, c_void_p, c_int, ctypes.POINTER(c_int), c_int,
                                         c_int, c_void_p, c_size_t, c_void_p]),
        "ve_circulant_project_noalloc": (c_int, [c_void_p, c_void_p, c_int, ctypes.POINTER(c_int),
                                                 c_int, c_int, c_void_p]),
        "ve_general_create": (c_int, [ctypes.POINTER(ve_terms), c_int, ctypes.POINTER(ve_options),
                                      ctypes.POINTER(c_void_p)]),
        "ve_general_create_fermions": (c_int, [ctypes.POINTER(ve_fermion_terms), c_int,
                                               ctypes.POINTER(ve_options), ctypes.POINTER(c_void_p)]),
        "ve_spin_blocks": (c_int, [ctypes.POINTER(ve_terms), c_int, P_double, P_double]),
        "ve_fermion_blocks": (c_int, [ctypes.POINTER(ve_fermion_terms), c_int, P_double, P_double]),
        "ve_general_destroy": (None, [c_void_p]),
        "ve_general_dims": (c_int, [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                    ctypes.POINTER(c_int), ctypes.POINTER(c_long)]),
        "ve_general_iterate": (c_int, [c_void_p, c_long, c_double, ctypes.POINTER(ve_status)]),
        "ve_general_get_status": (c_int, [c_void_p, ctypes.POINTER(ve_status)]),
        "ve_general_bound": (c_int, [c_void_p, ctypes.POINTER(ve_cert)]),
        "ve_general_state_size": (c_size_t, [c_void_p]),
        "ve_general_get_state": (c_int, [c_void_p, P_double, c_size_t]),
        "ve_general_set_state": (c_int, [c_void_p, P_double, c_size_t]),
        "ve_general_profile": (c_int, [c_void_p, c_int]),
        "ve_general_profile_read": (c_int, [c_void_p, P_double, ctypes.POINTER(c_long), P_double]),
        "ve_general_profile_rounds": (c_int, [c_void_p, P_double, ctypes.POINTER(c_long),
                                              ctypes.POINTER(c_long)]),
        "ve_project_psd_dense_workspace_size": (c_size_t, [c_int]),
        "ve_project_psd_dense": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_size_t,
                                         c_void_p, ctypes.POINTER(c_int)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
lib = _lib


def _check(code, where):
    if code < 0:
        raise VEError(code, where)
    return code


def ve_error_string(code):
    return _lib.ve_error_string(int(code)).decode()


def ve_default_options(**overrides):
    opt = ve_options()
    _lib.ve_default_options(ctypes.byref(opt))
    for k, v in overrides.items():
        setattr(opt, k, v)
    return opt


def ve_ham_tfim(dim, J, h):
    out = ve_hamiltonian()
    _check(_lib.ve_ham_tfim(int(dim), float(J), float(h), ctypes.byref(out)), "ve_ham_tfim")
    return out


def ve_ham_xxz(dim, J, delta):
    out = ve_hamiltonian()
    _check(_lib.ve_ham_xxz(int(dim), float(J), float(delta), ctypes.byref(out)), "ve_ham_xxz")
    return out


def make_lattice(extent):
    extent = tuple(int(e) for e in extent)
    lat = ve_lattice()
    lat.dim = len(extent)
    for i, e in enumerate(extent):
        lat.extent[i] = e
    return lat


def make_cluster(extent):
    extent = tuple(int(e) for e in extent)
    clu = ve_cluster()
    for i, e in enumerate(extent):
        clu.extent[i] = e
    if len(extent) == 1:
        clu.extent[1] = 1
    return clu


def ve_create(lattice, cluster, ham, opt=None):
    """lattice / cluster: ve_lattice / ve_cluster or tuples of extents.  Returns a handle (int)."""
    if not isinstance(lattice, ve_lattice):
        lattice = make_lattice(lattice)
    if not isinstance(cluster, ve_cluster):
        cluster = make_cluster(cluster)
    h = c_void_p()
    _check(_lib.ve_create(ctypes.byref(lattice), ctypes.byref(cluster), ctypes.byref(ham),
                          ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)),
           "ve_create")
    return h.value


def ve_iterate(h, max_iter, tol=0.0):
    st = ve_status()
    code = _check(_lib.ve_iterate(c_void_p(h), int(max_iter), float(tol), ctypes.byref(st)),
                  "ve_iterate")
    return code, st


def ve_bound(h):
    c = ve_cert()
    _check(_lib.ve_bound(c_void_p(h), ctypes.byref(c)), "ve_bound")
    return c


def ve_destroy(h):
    _lib.ve_destroy(c_void_p(h) if h else None)


def ve_dims(h):
    N, m, D = c_int(), c_int(), c_int()
    _check(_lib.ve_dims(c_void_p(h), ctypes.byref(N), ctypes.byref(m), ctypes.byref(D)), "ve_dims")
    return N.value, m.value, D.value


def ve_state_size(h):
    return _lib.ve_state_size(c_void_p(h))


def ve_get_state(h, out=None):
    n = ve_state_size(h)
    if out is None:
        out = np.empty(n // 8, dtype=np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous
    _check(_lib.ve_get_state(c_void_p(h), out.ctypes.data_as(P_double), out.nbytes), "ve_get_state")
    return out


def ve_set_state(h, vec):
    vec = np.ascontiguousarray(vec, dtype=np.float64)
    _check(_lib.ve_set_state(c_void_p(h), vec.ctypes.data_as(P_double), vec.nbytes), "ve_set_state")


def ve_get_status(h):
    st = ve_status()
    _check(_lib.ve_get_status(c_void_p(h), ctypes.byref(st)), "ve_get_status")
    return st


def ve_profile(h, enable):
    _check(_lib.ve_profile(c_void_p(h), int(enable)), "ve_profile")


def ve_profile_read(h):
    ms = (c_double * VE_NSTAGE)()
    n = (c_long * VE_NSTAGE)()
    _check(_lib.ve_profile_read(c_void_p(h), ms, n), "ve_profile_read")
    return {STAGES[i]: (ms[i], n[i]) for i in range(VE_NSTAGE)}


def ve_profile_sweeps(h):
    a, b = c_double(), c_double()
    _check(_lib.ve_profile_sweeps(c_void_p(h), ctypes.byref(a), ctypes.byref(b)),
           "ve_profile_sweeps")
    return a.value, b.value


def ve_profile_first_order(h):
    """((first-order stops, eigensolves) of the pair projections, (same) of the wavevector
    projections) over the profiled sweeps."""
    p, k = (c_long * 2)(), (c_long * 2)()
    _check(_lib.ve_profile_first_order(c_void_p(h), p, k), "ve_profile_first_order")
    return (p[0], p[1]), (k[0], k[1])


def ve_selftest_bounded_wait():
    """Run the tensor-core kernels' timeout path once (loads withheld, then a clean call);
    returns the stalled call's device seconds.  Raises VEError on failure."""
    sec = c_double()
    _check(_lib.ve_selftest_bounded_wait(ctypes.byref(sec)), "ve_selftest_bounded_wait")
    return sec.value


def ve_project_psd_sym(in_ptr, out_ptr, n, count, precision=VE_PREC_FP64, stream=None):
    return _check(_lib.ve_project_psd_sym(in_ptr, out_ptr, int(n), int(count), int(precision),
                                          stream), "ve_project_psd_sym")


def ve_project_psd_herm(in_ptr, out_ptr, n, count, precision=VE_PREC_FP64, stream=None):
    return _check(_lib.ve_project_psd_herm(in_ptr, out_ptr, int(n), int(count), int(precision),
                                           stream), "ve_project_psd_herm")


def ve_project_psd_large_workspace_size(n, hermitian=False, precision=VE_PREC_FP64):
    return _lib.ve_project_psd_large_workspace_size(int(n), 1 if hermitian else 0, int(precision))


def ve_project_psd_sym_large(in_ptr, out_ptr, n, count, ws_ptr, ws_bytes, precision=VE_PREC_FP64,
                             stream=None):
    return _check(_lib.ve_project_psd_sym_large(in_ptr, out_ptr, int(n), int(count),
                                                int(precision), ws_ptr, int(ws_bytes), stream),
                  "ve_project_psd_sym_large")


def ve_project_psd_herm_large(in_ptr, out_ptr, n, count, ws_ptr, ws_bytes, precision=VE_PREC_FP64,
                              stream=None):
    return _check(_lib.ve_project_psd_herm_large(in_ptr, out_ptr, int(n), int(count),
                                                 int(precision), ws_ptr, int(ws_bytes), stream),
                  "ve_project_psd_herm_large")


def _M(M):
    M = tuple(int(x) for x in M)
    arr = (c_int * 2)(M[0], M[1] if len(M) > 1 else 1)
    return len(M), arr


def ve_circulant_workspace_size(M, D):
    dim, arr = _M(M)
    return _lib.ve_circulant_workspace_size(dim, arr, int(D))


def ve_circulant_project(x_in_ptr, x_out_ptr, M, D, workspace_ptr, workspace_bytes,
                         precision=VE_PREC_FP64, stream=None):
    dim, arr = _M(M)
    return _check(_lib.ve_circulant_project(x_in_ptr, x_out_ptr, dim, arr, int(D), int(precision),
                                            workspace_ptr, int(workspace_bytes), stream),
                  "ve_circulant_project")


def ve_circulant_project_noalloc(x_in_ptr, x_out_ptr, M, D, precision=VE_PREC_FP64, stream=None):
    """The X step with the library's fixed scratch array (no allocation; see include/ve.h)."""
    dim, arr = _M(M)
    return _check(_lib.ve_circulant_project_noalloc(x_in_ptr, x_out_ptr, dim, arr, int(D),
                                                    int(precision), stream),
                  "ve_circulant_project_noalloc")


def ve_create_batch(instances, opt=None):
    """instances: list of (lattice extents, cluster extents, ve_hamiltonian).  Returns a batch."""
    n = len(instances)
    lats = (ve_lattice * n)(*[make_lattice(l) for l, _, _ in instances])
    clus = (ve_cluster * n)(*[make_cluster(c) for _, c, _ in instances])
    hams = (ve_hamiltonian * n)(*[hm for _, _, hm in instances])
    b = c_void_p()
    _check(_lib.ve_create_batch(n, lats, clus, hams, ctypes.byref(opt) if opt is not None else None,
                                ctypes.byref(b)), "ve_create_batch")
    return b.value


def ve_batch_size(b):
    return _lib.ve_batch_size(c_void_p(b))


def ve_batch_handle(b, i):
    return _lib.ve_batch_handle(c_void_p(b), int(i))


def ve_batch_iterate(b, max_iter, tol=0.0):
    n = ve_batch_size(b)
    st = (ve_status * n)()
    code = _check(_lib.ve_batch_iterate(c_void_p(b), int(max_iter), float(tol), st),
                  "ve_batch_iterate")
    return code, list(st)


def ve_batch_bound(b):
    n = ve_batch_size(b)
    c = (ve_cert * n)()
    _check(_lib.ve_batch_bound(c_void_p(b), c), "ve_batch_bound")
    return list(c)


def ve_batch_destroy(b):
    _lib.ve_batch_destroy(c_void_p(b) if b else None)


def ve_project_state_x(h):
    _check(_lib.ve_project_state_x(c_void_p(h)), "ve_project_state_x")


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(P_float)


def ve_mlp_create(n_in, n_hidden, n_layers, n_out, seed=20210604):
    m = c_void_p()
    _check(_lib.ve_mlp_create(int(n_in), int(n_hidden), int(n_layers), int(n_out), int(seed),
                              ctypes.byref(m)), "ve_mlp_create")
    return m.value


def ve_mlp_destroy(m):
    _lib.ve_mlp_destroy(c_void_p(m) if m else None)


def ve_mlp_num_params(m):
    return _lib.ve_mlp_num_params(c_void_p(m))


def ve_mlp_get_params(m):
    out = np.empty(ve_mlp_num_params(m), dtype=np.float32)
    _check(_lib.ve_mlp_get_params(c_void_p(m), out.ctypes.data_as(P_float), out.size), "ve_mlp_get_params")
    return out


def ve_mlp_set_params(m, params):
    p, pp = _f32(params)
    _check(_lib.ve_mlp_set_params(c_void_p(m), pp, p.size), "ve_mlp_set_params")


def ve_mlp_loss_grad(m, x, t):
    x, xp = _f32(x)
    t, tp = _f32(t)
    loss = ctypes.c_float()
    g = np.empty(ve_mlp_num_params(m), dtype=np.float32)
    _check(_lib.ve_mlp_loss_grad(c_void_p(m), xp, tp, x.shape[0], ctypes.byref(loss),
                                 g.ctypes.data_as(P_float)), "ve_mlp_loss_grad")
    return loss.value, g


def ve_mlp_train(m, x, t, steps, lr=1e-3):
    x, xp = _f32(x)
    t, tp = _f32(t)
    loss = ctypes.c_float()
    _check(_lib.ve_mlp_train(c_void_p(m), xp, tp, x.shape[0], int(steps), float(lr),
                             ctypes.byref(loss)), "ve_mlp_train")
    return loss.value


def ve_mlp_predict(m, x, n_out):
    x, xp = _f32(x)
    y = np.empty((x.shape[0], n_out), dtype=np.float32)
    _check(_lib.ve_mlp_predict(c_void_p(m), xp, x.shape[0], y.ctypes.data_as(P_float)),
           "ve_mlp_predict")
    return y


# ---- general Hamiltonians (Algorithm 5) ------------------------------------------------------
def _spin_terms(terms):
    """ve_terms for dict(nspins, onsite (nspins, 2, 2) or None, bond_sites (nb, 2),
    bond_ops (nb, 4, 4)); the arrays it points to are returned with it to keep them alive."""
    nspins = int(terms["nspins"])
    onsite = terms.get("onsite")
    on = None if onsite is None else np.ascontiguousarray(onsite, dtype=np.float64).reshape(nspins, 4)
    sites = np.ascontiguousarray(terms["bond_sites"], dtype=np.int32).reshape(-1, 2)
    ops = np.ascontiguousarray(terms["bond_ops"], dtype=np.float64).reshape(-1, 16)
    t = ve_terms(nspins, on.ctypes.data if on is not None else None, sites.shape[0],
                 sites.ctypes.data if sites.size else None, ops.ctypes.data if ops.size else None)
    return t, (on, sites, ops)


def _fermion_terms(terms):
    """ve_fermion_terms for dict(nsites, hops [(i, j, t)], pairs [(i, j, v)])."""
    hops = list(terms.get("hops", ()))
    pairs = list(terms.get("pairs", ()))
    hs = np.ascontiguousarray([(i, j) for i, j, _ in hops], dtype=np.int32).reshape(-1, 2)
    ht = np.ascontiguousarray([t for _, _, t in hops], dtype=np.float64)
    ps = np.ascontiguousarray([(i, j) for i, j, _ in pairs], dtype=np.int32).reshape(-1, 2)
    pv = np.ascontiguousarray([v for _, _, v in pairs], dtype=np.float64)
    t = ve_fermion_terms(int(terms["nsites"]), len(hops), hs.ctypes.data if hops else None,
                         ht.ctypes.data if hops else None, len(pairs),
                         ps.ctypes.data if pairs else None, pv.ctypes.data if pairs else None)
    return t, (hs, ht, ps, pv)


def ve_general_create(terms, cluster_spins, opt=None):
    """terms: dict(nspins, onsite (nspins, 2, 2) or None, bond_sites (nb, 2), bond_ops (nb, 4, 4)).
    Returns a handle (int)."""
    t, keep = _spin_terms(terms)
    h = c_void_p()
    _check(_lib.ve_general_create(ctypes.byref(t), int(cluster_spins),
                                  ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)),
           "ve_general_create")
    return h.value


def _blocks(fn, t, n_units, L, name):
    m = 2 ** L
    N = n_units // L
    K = N * (N - 1) // 2
    Hi = np.zeros((N, m, m))
    Hij = np.zeros((K, m * m, m * m))
    _check(fn(ctypes.byref(t), int(L), Hi.ctypes.data_as(P_double), Hij.ctypes.data_as(P_double)),
           name)
    return Hi, Hij


def ve_spin_blocks(terms, cluster_spins):
    """(Hi (N, m, m), Hij (K, D, D)) that ve_general_create builds, on the host."""
    t, keep = _spin_terms(terms)
    return _blocks(_lib.ve_spin_blocks, t, int(terms["nspins"]), cluster_spins, "ve_spin_blocks")


def ve_fermion_blocks(terms, cluster_sites):
    """(Hi, Hij) that ve_general_create_fermions builds, on the host."""
    t, keep = _fermion_terms(terms)
    return _blocks(_lib.ve_fermion_blocks, t, int(terms["nsites"]), cluster_sites,
                   "ve_fermion_blocks")


def ve_general_create_fermions(terms, cluster_sites, opt=None):
    """terms: dict(nsites, hops [(i, j, t)], pairs [(i, j, v)]).  Returns a handle (int)."""
    t, keep = _fermion_terms(terms)
    h = c_void_p()
    _check(_lib.ve_general_create_fermions(ctypes.byref(t), int(cluster_sites),
                                           ctypes.byref(opt) if opt is not None else None,
                                           ctypes.byref(h)), "ve_general_create_fermions")
    return h.value


def ve_general_destroy(h):
    _lib.ve_general_destroy(c_void_p(h) if h else None)


def ve_general_dims(h):
    N, m, D, K = c_int(), c_int(), c_int(), c_long()
    _check(_lib.ve_general_dims(c_void_p(h), ctypes.byref(N), ctypes.byref(m), ctypes.byref(D),
                                ctypes.byref(K)), "ve_general_dims")
    return N.value, m.value, D.value, K.value


def ve_general_iterate(h, max_iter, tol=0.0):
    st = ve_status()
    code = _check(_lib.ve_general_iterate(c_void_p(h), int(max_iter), float(tol), ctypes.byref(st)),
                  "ve_general_iterate")
    return code, st


def ve_general_get_status(h):
    st = ve_status()
    _check(_lib.ve_general_get_status(c_void_p(h), ctypes.byref(st)), "ve_general_get_status")
    return st


def ve_general_bound(h):
    c = ve_cert()
    _check(_lib.ve_general_bound(c_void_p(h), ctypes.byref(c)), "ve_general_bound")
    return c


def ve_general_state_size(h):
    return _lib.ve_general_state_size(c_void_p(h))


def ve_general_get_state(h, out=None):
    n = ve_general_state_size(h)
    if out is None:
        out = np.empty(n // 8, dtype=np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous
    _check(_lib.ve_general_get_state(c_void_p(h), out.ctypes.data_as(P_double), out.nbytes),
           "ve_general_get_state")
    return out


def ve_general_set_state(h, vec):
    vec = np.ascontiguousarray(vec, dtype=np.float64)
    _check(_lib.ve_general_set_state(c_void_p(h), vec.ctypes.data_as(P_double), vec.nbytes),
           "ve_general_set_state")


def ve_general_profile(h, enable):
    _check(_lib.ve_general_profile(c_void_p(h), int(enable)), "ve_general_profile")


def ve_general_profile_read(h):
    ms = (c_double * VE_GENERAL_NSTAGE)()
    nl = (c_long * VE_GENERAL_NSTAGE)()
    sw = c_double()
    _check(_lib.ve_general_profile_read(c_void_p(h), ms, nl, ctypes.byref(sw)),
           "ve_general_profile_read")
    return list(ms), list(nl), sw.value


def ve_general_profile_rounds(h):
    """(ms of the profiled Jacobi sweeps, round launches in them, X steps ended first-order)."""
    ms, r, fo = c_double(), c_long(), c_long()
    _check(_lib.ve_general_profile_rounds(c_void_p(h), ctypes.byref(ms), ctypes.byref(r),
                                          ctypes.byref(fo)), "ve_general_profile_rounds")
    return ms.value, r.value, fo.value


def ve_project_psd_dense_workspace_size(n):
    return _lib.ve_project_psd_dense_workspace_size(int(n))


VE_DENSE_WARM = 1
VE_DENSE_FIRST_ORDER = 2


def ve_project_psd_dense(in_ptr, out_ptr, n, ws_ptr, ws_bytes, warm=0, stream=None,
                         first_order=False):
    """Returns the Jacobi sweeps taken (+1000 when the first-order reconstruction ended them)."""
    sw = c_int()
    flags = (VE_DENSE_WARM if warm else 0) | (VE_DENSE_FIRST_ORDER if first_order else 0)
    _check(_lib.ve_project_psd_dense(c_void_p(in_ptr), c_void_p(out_ptr), int(n), flags,
                                     c_void_p(ws_ptr), int(ws_bytes), c_void_p(stream),
                                     ctypes.byref(sw)), "ve_project_psd_dense")
    return sw.value
