"""The C-ABI library loads, exports every symbol include/ve.h declares, and its host-only entry
points (no GPU work) behave as documented.  No kernel is launched here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import __graft_entry__
from oracle import models as mo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ve.h")


@pytest.fixture(scope="module")
def ve():
    __graft_entry__.build()
    from paper_2106_02682_gb300 import ve as mod
    return mod


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ve_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(ve):
    names = declared_functions()
    assert len(names) >= 17
    out = subprocess.run(["nm", "-D", "--defined-only", ve.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(ve_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(ve.lib, n)


def test_struct_layouts_match_the_header(ve, tmp_path):
    """Compile a C probe against include/ve.h and compare sizes/offsets with the ctypes mirror."""
    structs = {"ve_lattice": ve.ve_lattice, "ve_cluster": ve.ve_cluster,
               "ve_hamiltonian": ve.ve_hamiltonian, "ve_options": ve.ve_options,
               "ve_status": ve.ve_status, "ve_cert": ve.ve_cert, "ve_terms": ve.ve_terms,
               "ve_fermion_terms": ve.ve_fermion_terms}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ve.h"', 'int main(void){']
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.splitlines():
        name, field, val = line.split()
        cls = structs[name]
        if field == "size":
            assert ctypes.sizeof(cls) == int(val), name
        else:
            assert getattr(cls, field).offset == int(val), (name, field)


def test_defaults_and_error_strings(ve):
    opt = ve.ve_default_options()
    assert (opt.mu, opt.nu, opt.eps, opt.precision, opt.check_every) == (10.0, 10.0, 2.0, 0, 10)
    assert opt.stream is None
    for code in (0, 1, -1, -2, -3, -4, -5, -6):
        assert ve.ve_error_string(code) and ve.ve_error_string(code) != "unknown status"
    assert ve.ve_error_string(42) == "unknown status"


@pytest.mark.parametrize("dim", [1, 2])
def test_site_terms_match_the_oracle_models(ve, dim):
    for J, h in [(1.0, 0.5), (0.7, 1.3)]:
        H = ve.ve_ham_tfim(dim, J, h)
        on, bonds = mo.tfim_terms(J, h, dim)
        np.testing.assert_array_equal(np.array(H.onsite).reshape(2, 2), on)
        assert H.nbond == dim
        for b, (off, B) in enumerate(bonds):
            np.testing.assert_array_equal(np.array(H.bond[b]).reshape(4, 4), B)
            assert tuple(H.bond_offset[b])[:dim] == off
    for J, d in [(1.0, 1.0), (0.5, 0.3)]:
        H = ve.ve_ham_xxz(dim, J, d)
        on, bonds = mo.xxz_terms(J, d, dim)
        np.testing.assert_allclose(np.array(H.bond[0]).reshape(4, 4), bonds[0][1], atol=1e-15)
    with pytest.raises(ve.VEError):
        ve.ve_ham_tfim(3, 1.0, 1.0)


@pytest.mark.parametrize("lattice,cluster,code", [
    ((8,), (3,), -1),          # cluster does not tile the lattice
    ((2,), (2,), -1),          # a single cluster (N < 2)
    ((20,), (5,), -5),         # 5-spin clusters (D = 1024): not built here
    ((4 * 67,), (1,), -5),     # N = 268 > 64 does not split into two factors <= 64
    ((8000,), (1,), -5),       # N > 4096
    ((130, 4), (1, 1), -5),    # 2-D axis with more than 64 clusters
])
def test_create_rejects_bad_shapes_before_touching_the_gpu(ve, lattice, cluster, code):
    with pytest.raises(ve.VEError) as ei:
        ve.ve_create(lattice, cluster, ve.ve_ham_tfim(len(lattice), 1.0, 1.0))
    assert ei.value.code == code


def test_create_rejects_bad_options(ve):
    for bad in (dict(mu=0.0), dict(nu=-1.0), dict(eps=0.0), dict(check_every=0), dict(precision=7)):
        with pytest.raises(ve.VEError) as ei:
            ve.ve_create((8,), (1,), ve.ve_ham_tfim(1, 1.0, 1.0), ve.ve_default_options(**bad))
        assert ei.value.code == -1


def test_null_handles_are_rejected(ve):
    assert ve.lib.ve_iterate(None, 1, 0.0, None) == -1
    assert ve.lib.ve_bound(None, None) == -1
    assert ve.lib.ve_state_size(None) == 0
    ve.ve_destroy(None)
    assert ve.ve_circulant_workspace_size((3, 5), 16) > 0
    assert ve.ve_circulant_workspace_size((4 * 67,), 16) == 0


def _terms(nspins, bonds=((0, 1),)):
    sites = np.array(bonds, dtype=np.int32).reshape(-1, 2)
    return dict(nspins=nspins, onsite=np.zeros((nspins, 2, 2)), bond_sites=sites,
                bond_ops=np.zeros((len(sites), 4, 4)))


@pytest.mark.parametrize("nspins,L,bonds,code", [
    (8, 4, ((0, 1),), -5),         # 4-spin clusters: not built for the general solver
    (7, 2, ((0, 1),), -1),         # clusters do not tile the spins
    (2, 2, ((0, 1),), -1),         # a single cluster
    (260, 1, ((0, 1),), -5),       # N D = 1040 > 1024: beyond the dense X step
    (4, 1, ((2, 2),), -1),         # a bond on one spin
    (4, 1, ((0, 4),), -1),         # a spin out of range
])
def test_general_create_rejects_bad_terms_before_touching_the_gpu(ve, nspins, L, bonds, code):
    with pytest.raises(ve.VEError) as ei:
        ve.ve_general_create(_terms(nspins, bonds), L)
    assert ei.value.code == code


def test_general_create_rejects_other_precisions_and_bad_options(ve):
    for bad, code in ((dict(precision=ve.VE_PREC_MIXED), -5), (dict(mu=0.0), -1),
                      (dict(check_every=0), -1)):
        with pytest.raises(ve.VEError) as ei:
            ve.ve_general_create(_terms(4), 1, ve.ve_default_options(**bad))
        assert ei.value.code == code


def test_general_null_handles_and_dense_workspace_sizes(ve):
    assert ve.lib.ve_general_iterate(None, 1, 0.0, None) == -1
    assert ve.lib.ve_general_bound(None, None) == -1
    assert ve.lib.ve_general_state_size(None) == 0
    assert ve.lib.ve_general_dims(None, None, None, None, None) == -1
    ve.ve_general_destroy(None)
    for n, ok in ((2, True), (24, True), (512, True), (1024, True), (511, False), (1026, False),
                  (0, False)):
        assert (ve.ve_project_psd_dense_workspace_size(n) > 0) == ok, n
    # two n x n float64 matrices plus small vectors
    assert ve.ve_project_psd_dense_workspace_size(512) >= 2 * 512 * 512 * 8


@pytest.mark.parametrize("nspins,L,kind", [(6, 1, "tfim"), (8, 2, "xxz"), (9, 3, "tfim")])
def test_host_spin_blocks_match_the_oracle(ve, nspins, L, kind):
    from oracle import models
    from paper_2106_02682_gb300 import synth
    terms = synth.disordered_chain(nspins, kind, alpha=1.5, seed=nspins)
    bonds = [(int(s), int(t), B) for (s, t), B in zip(terms['bond_sites'], terms['bond_ops'])]
    ref = models.general_blocks(nspins, L, terms['onsite'], bonds)
    Hi, Hij = ve.ve_spin_blocks(terms, L)
    np.testing.assert_allclose(Hi, ref['Hi'], atol=1e-14)
    np.testing.assert_allclose(Hij, ref['Hij'], atol=1e-14)


@pytest.mark.parametrize("M,L,U,lr", [(6, 1, 1.5, False), (8, 2, 2.0, False), (8, 2, 1.0, True),
                                      (9, 3, 0.7, True), (12, 2, 0.0, False)])
def test_host_fermion_blocks_match_the_oracle(ve, M, L, U, lr):
    # the library enumerates basis states with explicit string signs, the oracle multiplies
    # Kronecker-product creation operators: two independent Jordan-Wigner constructions
    from oracle import fermions
    from paper_2106_02682_gb300 import synth
    terms = synth.fermion_ring(M, U, long_range=lr)
    oh, op = fermions.ring_terms(M, U, long_range=lr)
    assert [tuple(x) for x in terms['hops']] == [tuple(x) for x in oh]
    assert [tuple(x) for x in terms['pairs']] == pytest.approx([tuple(x) for x in op])
    ref = fermions.fermion_blocks(M, L, U, long_range=lr)
    Hi, Hij = ve.ve_fermion_blocks(terms, L)
    np.testing.assert_allclose(Hi, ref['Hi'], atol=1e-14)
    np.testing.assert_allclose(Hij, ref['Hij'], atol=1e-14)


def test_fermion_create_rejects_bad_terms_before_touching_the_gpu(ve):
    for terms, L, code in ((dict(nsites=8, hops=[(0, 0, -1.0)]), 2, -1),
                           (dict(nsites=8, hops=[(0, 8, -1.0)]), 2, -1),
                           (dict(nsites=7, hops=[(0, 1, -1.0)]), 2, -1),
                           (dict(nsites=8, hops=[(0, 1, -1.0)]), 4, -5),
                           (dict(nsites=272, hops=[(0, 1, -1.0)]), 1, -5)):
        with pytest.raises(ve.VEError) as ei:
            ve.ve_general_create_fermions(terms, L)
        assert ei.value.code == code
