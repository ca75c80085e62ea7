"""The allocation-free X step (ve_circulant_project_noalloc) against the oracle and against the
allocating entry point.

Some callers may not allocate device memory (a plugin whose framework owns every allocation, a
latency-critical loop that must not hit cudaMalloc's synchronisation).  The no-allocation entry
point serves them from a fixed scratch array inside the library.  Through the C ABI, in every
arithmetic, this test checks two calls in a row -- a large first block row, then a different
smaller one, so that the second call runs over the first call's leftovers in the shared array --
against the oracle's block-DFT projection and against ve_circulant_project with a caller-provided
workspace, one call with the output aliasing the input, and that requests above the fixed size
are refused.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import __graft_entry__
from oracle import ve_oracle as vo
from paper_2106_02682_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# The tolerances of the X-step parity test: float64 1e-10 relative to the largest entry,
# double-float 32 times that (the ratio of the unit roundoffs 2^-48 / 2^-53), float32 2e-4.
TOL = {0: 1e-10, 1: 2e-4, 2: 1e-10 * 32}


@pytest.fixture(scope="module")
def ve():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    __graft_entry__.build()
    from paper_2106_02682_gb300 import ve as mod
    return mod


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def _oracle(X, M):
    return np.real(vo._lattice_dft(vo.proj_psd(vo._lattice_dft(X, M, False)), M, True))


def _allocating(ve, X, M, D, prec):
    ws_bytes = ve.ve_circulant_workspace_size(M, D)
    ws = torch.empty(ws_bytes // 8 + 64, dtype=torch.float64, device="cuda")
    x = torch.from_numpy(X).cuda()
    y = torch.empty_like(x)
    ve.ve_circulant_project(x.data_ptr(), y.data_ptr(), M, D, ws.data_ptr(), ws_bytes, prec)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 2, 1])
def test_noalloc_matches_oracle_and_allocating_entry_point_on_consecutive_calls(ve, prec):
    for M, D, seed in [((4096,), 16, 11), ((8, 6), 16, 12)]:
        X = synth.circulant_first_row(M, D, seed=seed)
        ref = _oracle(X, M)
        alloc = _allocating(ve, X, M, D, prec)
        x = torch.from_numpy(X).cuda()
        y = torch.full_like(x, np.nan)
        ve.ve_circulant_project_noalloc(x.data_ptr(), y.data_ptr(), M, D, prec)
        torch.cuda.synchronize()
        out = y.cpu().numpy()
        assert _relerr(out, ref) <= TOL[prec], (M, D, prec, _relerr(out, ref))
        assert _relerr(out, alloc) <= TOL[prec], (M, D, prec, _relerr(out, alloc))


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_in_place(ve, prec):
    """Output aliasing the input, as include/ve.h allows: the same result as a separate output."""
    M, D = (50,), 16
    X = synth.circulant_first_row(M, D, seed=13)
    x = torch.from_numpy(X).cuda()
    y = torch.empty_like(x)
    ve.ve_circulant_project_noalloc(x.data_ptr(), y.data_ptr(), M, D, prec)
    ve.ve_circulant_project_noalloc(x.data_ptr(), x.data_ptr(), M, D, prec)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    assert _relerr(y.cpu().numpy(), _oracle(X, M)) <= TOL[prec]


def test_noalloc_refuses_requests_above_its_scratch(ve):
    M, D = (64, 64), 64          # N D^2 = 2^24 entries, far above the fixed array
    assert ve.ve_circulant_workspace_size(M, D) > ve.VE_NOALLOC_SCRATCH_BYTES
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ve.VEError) as ei:
        ve.ve_circulant_project_noalloc(x.data_ptr(), x.data_ptr(), M, D, 0)
    assert ei.value.code == ve.VE_EINVAL
