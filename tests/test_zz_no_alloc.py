"""The allocation-free X step (ve_circulant_project_noalloc) against the allocating one.

Some callers may not allocate device memory (a plugin whose framework owns every allocation, a
latency-critical loop that must not hit cudaMalloc's synchronisation).  The no-allocation entry
point serves them from a fixed scratch array inside the library; this test checks, through the
C ABI, that two calls in a row -- a large first block row, then a different smaller one, so that
the second call runs over the first call's leftovers in the shared array -- give the same result
as ve_circulant_project with a caller-provided workspace, and that requests above the fixed size
are refused.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import __graft_entry__
from paper_2106_02682_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL64 = 1e-10   # the float64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def ve():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    __graft_entry__.build()
    from paper_2106_02682_gb300 import ve as mod
    return mod


def _allocating(ve, X, M, D):
    ws_bytes = ve.ve_circulant_workspace_size(M, D)
    ws = torch.empty(ws_bytes // 8 + 64, dtype=torch.float64, device="cuda")
    x = torch.from_numpy(X).cuda()
    y = torch.empty_like(x)
    ve.ve_circulant_project(x.data_ptr(), y.data_ptr(), M, D, ws.data_ptr(), ws_bytes, 0)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def test_noalloc_matches_the_allocating_entry_point_on_consecutive_calls(ve):
    for M, D, seed in [((4096,), 16, 11), ((8, 6), 16, 12)]:
        X = synth.circulant_first_row(M, D, seed=seed)
        ref = _allocating(ve, X, M, D)
        x = torch.from_numpy(X).cuda()
        y = torch.full_like(x, np.nan)
        ve.ve_circulant_project_noalloc(x.data_ptr(), y.data_ptr(), M, D, 0)
        torch.cuda.synchronize()
        out = y.cpu().numpy()
        err = np.max(np.abs(out - ref)) / max(1.0, np.max(np.abs(ref)))
        assert err <= RTOL64, (M, D, err)


def test_noalloc_refuses_requests_above_its_scratch(ve):
    M, D = (64, 64), 64          # N D^2 = 2^24 entries, far above the fixed array
    assert ve.ve_circulant_workspace_size(M, D) > ve.VE_NOALLOC_SCRATCH_BYTES
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ve.VEError) as ei:
        ve.ve_circulant_project_noalloc(x.data_ptr(), x.data_ptr(), M, D, 0)
    assert ei.value.code == ve.VE_EINVAL
