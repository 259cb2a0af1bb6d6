"""The allocation-free moment limiter (lxw_moment_limit_noalloc) against the
solver-based one (lxw_moment_limit), through the C ABI.

Callers that cannot call cudaMalloc -- code whose device memory belongs to
another allocator (a caching pool or a fixed budget), code that must avoid
cudaMalloc's implicit synchronisation -- use the no-alloc form; its scratch
is a static device array shared by all calls, so the tests make calls in a
row (also a large call using three scratch slots followed by a one-slot
call) and check each against the existing entry point, and check the
non-positive-average status against the oracle's flattened cells.  This
file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
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
        L._check(L.lib().lxw_moment_limit_noalloc(0, 2, 16777217, 1.4, 1e-12, L._ptr(Q), None, L._ptr(s), None, None))
    assert e.value.code == L.ERR_ARG and "16777216" in str(e.value)
    with pytest.raises(L.LxwError):            # degree 4 is not provided
        L._check(L.lib().lxw_moment_limit_noalloc(0, 4, 4, 1.4, 1e-12, L._ptr(Q), None, L._ptr(s), None, None))


def _solver_limit(L, sol, Q0):
    N = Q0.shape[0]
    A = torch.from_numpy(Q0.copy()).cuda()
    tA = torch.zeros(N, dtype=torch.float64, device="cuda")
    sA = torch.zeros(1, dtype=torch.float64, device="cuda")
    L.lxw_moment_limit(sol, A, tA, sA)
    torch.cuda.synchronize()
    return A.cpu().numpy(), tA.cpu().numpy(), sA.item()


def test_noalloc_three_slots_then_one(L):
    """70,000 elements use three 32,768-element scratch slots; the next call
    (1,000 elements, one slot) must see only its own slot's maximum."""
    for n, seed, amp in ((265, 31, 1.0), (32, 32, 0.1)):      # 70,225 then 1,024 squares
        mesh = L.lxw_mesh_cartesian(n, n, bc=(2, 2, 2, 2))
        sol = L.lxw_solver_create(mesh, 2, stream=torch.cuda.current_stream())
        Q0 = synth.random_modal_state(sol.N, sol.ML, seed=seed, amp=amp)
        if n == 265:
            Q0[5, 3, 0] *= 100.0                               # the hottest (fastest) cell sits in slot 0
        QA, tA, sA = _solver_limit(L, sol, Q0)
        B = torch.from_numpy(Q0.copy()).cuda()
        tB = torch.zeros(sol.N, dtype=torch.float64, device="cuda")
        sB = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        L.lxw_moment_limit_noalloc(0, 2, B, tB, sB, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert np.abs(B.cpu().numpy() - QA).max() <= 1e-13 * np.abs(Q0).max()
        assert np.abs(tB.cpu().numpy() - tA).max() <= 1e-12
        assert abs(sB.item() - sA) <= 1e-14 * sA


def test_noalloc_reports_nonpositive_averages_like_the_oracle(L):
    """Cells with a non-positive average density or pressure: the oracle
    zeroes their higher modes (theta = 0) and flags them; the no-alloc call
    does the same, returns LXW_ERR_NONPOSITIVE without a status pointer and
    sets the bit with one; a clean call afterwards reports nothing."""
    from oracle import oracle as orc
    n = 12
    Q0 = synth.random_modal_state(n * n, 6, seed=77, amp=0.5)
    Q0[7, 0, 0] = -1e-3                                     # negative density
    Q0[30, 3, 0] = 0.2 * (0.5 * Q0[30, 1, 0] ** 2 / Q0[30, 0, 0])   # kinetic energy above E: p < 0
    osol = orc.Solver(orc.Mesh.cartesian(n, n), 2)
    Qo = Q0.copy()
    to, st = osol.moment_limit(Qo)
    assert st & 1 and to[7] == 0.0 and to[30] == 0.0
    B = torch.from_numpy(Q0.copy()).cuda()
    tB = torch.full((n * n,), -1.0, dtype=torch.float64, device="cuda")
    sB = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LxwError) as e:
        L.lxw_moment_limit_noalloc(0, 2, B, tB, sB, stream=torch.cuda.current_stream())
    assert e.value.code == L.ERR_NONPOSITIVE
    assert np.abs(B.cpu().numpy() - Qo).max() <= 1e-13 * np.abs(Q0).max()
    assert np.abs(tB.cpu().numpy() - to).max() <= 1e-12
    # with a status pointer: asynchronous, the bit lands on the device
    B = torch.from_numpy(Q0.copy()).cuda()
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    L.lxw_moment_limit_noalloc(0, 2, B, None, sB, stream=torch.cuda.current_stream(), status=status)
    torch.cuda.synchronize()
    assert status.item() == L.ST_NONPOSITIVE
    # the next clean call starts from a cleared status word
    C = torch.from_numpy(synth.random_modal_state(n * n, 6, seed=78, amp=0.5)).cuda()
    L.lxw_moment_limit_noalloc(0, 2, C, None, sB, stream=torch.cuda.current_stream(), status=status)
    torch.cuda.synchronize()
    assert status.item() == 0
    L.lxw_moment_limit_noalloc(0, 2, C, None, sB, stream=torch.cuda.current_stream())


def test_noalloc_checks_the_state_shape(L):
    """A P2 state passed with degree 3 (or a wrong variable count) is refused
    before anything runs on the device."""
    Q = torch.zeros((16, 4, 6), dtype=torch.float64, device="cuda")
    s = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LxwError) as e:
        L.lxw_moment_limit_noalloc(0, 3, Q, None, s)
    assert e.value.code == L.ERR_ARG and "[N][4][10]" in str(e.value)
    with pytest.raises(L.LxwError):
        L.lxw_moment_limit_noalloc(0, 2, torch.zeros((16, 3, 6), dtype=torch.float64, device="cuda"), None, s)
