"""The allocation-free moment limiter (lxw_moment_limit_noalloc) against the
solver-based one (lxw_moment_limit), through the C ABI.

Callers that cannot call cudaMalloc -- code running under stream capture,
code whose device memory belongs to another allocator, code that must avoid
cudaMalloc's implicit synchronisation -- use the no-alloc form; its scratch
is a static device array shared by all calls, so the test makes two calls in
a row and checks both against the existing entry point.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1601_08145_gb300 import build
    build.build()
    from paper_1601_08145_gb300 import lxw
    return lxw


@pytest.mark.parametrize("kind,deg,n", [(0, 2, 300), (1, 3, 90)])
def test_noalloc_matches_solver_moment_limiter_twice(L, kind, deg, n):
    if kind == 0:
        mesh = L.lxw_mesh_cartesian(n, n, bc=(2, 2, 2, 2))
    else:
        xy, tv = synth.structured_triangles(n, jitter=0.2, seed=4)
        mesh = L.lxw_mesh_triangles(xy, tv)
    sol = L.lxw_solver_create(mesh, deg, stream=torch.cuda.current_stream())
    N, ML = sol.N, sol.ML
    for call, seed in enumerate((11, 12)):           # two calls in a row, different inputs
        Q0 = synth.random_modal_state(N, ML, seed=seed, amp=1.2 if call == 0 else 0.4)
        Q0[::4, :, 1:] *= 0.05
        A = torch.from_numpy(Q0.copy()).cuda(); B = torch.from_numpy(Q0.copy()).cuda()
        tA = torch.zeros(N, dtype=torch.float64, device="cuda"); tB = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
        sA = torch.zeros(1, dtype=torch.float64, device="cuda"); sB = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        L.lxw_moment_limit(sol, A, tA, sA)
        L.lxw_moment_limit_noalloc(kind, deg, B, tB, sB, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert np.abs(B.cpu().numpy() - A.cpu().numpy()).max() <= 1e-13 * np.abs(Q0).max()
        assert np.abs(tB.cpu().numpy() - tA.cpu().numpy()).max() <= 1e-12
        assert abs(sB.item() - sA.item()) <= 1e-14 * sA.item()
        assert (tA.cpu().numpy() < 1).any()


def test_noalloc_rejects_bad_sizes(L):
    Q = torch.zeros((4, 4, 6), dtype=torch.float64, device="cuda")
    s = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LxwError) as e:       # beyond the static scratch capacity
        L._check(L.lib().lxw_moment_limit_noalloc(0, 2, 16777217, 1.4, 1e-12, L._ptr(Q), None, L._ptr(s), None))
    assert e.value.code == L.ERR_ARG and "16777216" in str(e.value)
    with pytest.raises(L.LxwError):            # degree 4 is not provided
        L._check(L.lib().lxw_moment_limit_noalloc(0, 4, 4, 1.4, 1e-12, L._ptr(Q), None, L._ptr(s), None))
