"""Batched independent problems (one solver over the disjoint union of the
meshes, persistent CTAs over a (problem, tile) work list, one graph per
step) against the same problems stepped one solver each.

Each problem's wave speed and time step are reductions over its own
elements (exact maxima), and every per-element computation is independent
of how elements are grouped into CTAs, so the batch must reproduce the
individual runs bit for bit, for every work-list configuration.
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


def quadrant_problem(L, n, seed):
    mesh = L.lxw_mesh_cartesian(n, n, (0.0, 1.0, 0.0, 1.0), (2, 2, 2, 2))
    return mesh, synth.ic_quadrants(seed)


def projected(L, sol, ic):
    xy = L.lxw_projection_points(sol)
    r, u, v, p = ic(xy[..., 0], xy[..., 1])
    prim = torch.from_numpy(np.stack(np.broadcast_arrays(r, u, v, p), axis=-1).copy()).cuda()
    Q = torch.zeros(sol.q64_shape, dtype=torch.float64, device="cuda")
    L.lxw_project(sol, prim, Q)
    return Q


@pytest.mark.parametrize("ctas,block,hi", [(0, 128, 0), (2, 128, 0), (1, 64, 1), (3, 32, 0)])
def test_batch_equals_individual_runs(L, ctas, block, hi):
    """hi: the high-occupancy kernel variants in the batch against the default
    variants one by one (the same arithmetic, other register budgets)."""
    sizes = [7, 13, 24, 5, 31]
    opt = L.lxw_options_default(precision=L.PREC_MIXED, ctas_per_sm=ctas, block_threads=block, high_occupancy=hi)
    probs = [quadrant_problem(L, n, 100 + k) for k, n in enumerate(sizes)]
    # individual solvers
    singles = []
    for mesh, ic in probs:
        s = L.lxw_solver_create(mesh, 2, L.lxw_options_default(precision=L.PREC_MIXED),
                                stream=torch.cuda.current_stream())
        st = L.new_state(s, projected(L, s, ic))
        for _ in range(12):
            L.lxw_step(s, st, 0.0, 0.3)
        singles.append(L.to_q64(s, st))
    # the batch
    b = L.lxw_batch_create([m for m, _ in probs], 2, opt, stream=torch.cuda.current_stream())
    Q = torch.cat([projected(L, L.lxw_solver_create(m, 2, stream=torch.cuda.current_stream()), ic)
                   for m, ic in probs])
    st = L.new_state(b, Q)
    L.lxw_run(b, st, 11, 0.3)
    d = L.lxw_step(b, st, 0.0, 0.3, diag=True)
    assert d["status"] == 0
    Qb = L.to_q64(b, st)
    torch.cuda.synchronize()
    off = b.offsets
    for k in range(len(sizes)):
        assert torch.equal(Qb[off[k]:off[k + 1]], singles[k]), k
    sv, dv = L.lxw_batch_scalars(b)
    assert len(sv) == len(sizes) and np.all(sv > 0) and len(set(np.round(dv, 15))) > 1


def test_autotune_keeps_results_and_restores_state(L):
    probs = [quadrant_problem(L, n, 7 + n) for n in (40, 17, 64, 9)]
    b = L.lxw_batch_create([m for m, _ in probs], 2, L.lxw_options_default(precision=L.PREC_MIXED),
                           stream=torch.cuda.current_stream())
    Q = torch.cat([projected(L, L.lxw_solver_create(m, 2, stream=torch.cuda.current_stream()), ic)
                   for m, ic in probs])
    A = L.new_state(b, Q)
    B = A.clone()
    L.lxw_run(b, A, 5, 0.3)
    res = L.lxw_autotune(b, B, 0.3, reps=2)
    torch.cuda.synchronize()
    assert torch.equal(B, L.new_state(b, Q))              # restored
    assert res["block_threads"] in (32, 64, 128) and res["ctas_per_sm"] in (0, 1, 2, 3, 4, 6, 8)
    assert res["high_occupancy"] in (0, 1)
    L.lxw_run(b, B, 5, 0.3)
    torch.cuda.synchronize()
    assert torch.equal(A, B)                              # the tuned configuration computes the same state


def test_ensemble_positivity(L):
    """A 24-problem ensemble of quadrant Riemann data stays positive."""
    sizes = synth.ensemble_sizes(24, 8, 40, seed=4242)
    probs = [quadrant_problem(L, int(n), 1000 + k) for k, n in enumerate(sizes)]
    b = L.lxw_batch_create([m for m, _ in probs], 2, L.lxw_options_default(precision=L.PREC_MIXED, ctas_per_sm=2),
                           stream=torch.cuda.current_stream())
    Q = torch.cat([projected(L, L.lxw_solver_create(m, 2, stream=torch.cuda.current_stream()), ic)
                   for m, ic in probs])
    st = L.new_state(b, Q)
    for _ in range(40):
        d = L.lxw_step(b, st, 0.0, 0.3, diag=True)
        assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0


def test_gated_batch_equals_gated_individual_runs(L):
    """The learned gate on a batch: its tensor-core tiles of 128 cells
    straddle problems, but every output row of the network depends only on its
    own cell, so the batch reproduces the problems gated one by one, bit for bit."""
    sizes = [9, 30, 17]
    net = L.lxw_mlp_create(256, seed=21, stream=torch.cuda.current_stream())
    probs = [quadrant_problem(L, n, 300 + k) for k, n in enumerate(sizes)]
    opt = L.lxw_options_default(precision=L.PREC_MIXED)
    singles = []
    for mesh, ic in probs:
        s = L.lxw_solver_create(mesh, 2, opt, stream=torch.cuda.current_stream())
        L.lxw_solver_set_mlp(s, net, 0.3)
        st = L.new_state(s, projected(L, s, ic))
        skipped = 0
        for _ in range(6):
            skipped += L.lxw_step(s, st, 0.0, 0.3, diag=True)["n_mlp_skip"]
        singles.append((L.to_q64(s, st), skipped))
    b = L.lxw_batch_create([m for m, _ in probs], 2, opt, stream=torch.cuda.current_stream())
    L.lxw_solver_set_mlp(b, net, 0.3)
    Q = torch.cat([projected(L, L.lxw_solver_create(m, 2, stream=torch.cuda.current_stream()), ic)
                   for m, ic in probs])
    st = L.new_state(b, Q)
    skipped = 0
    for _ in range(6):
        d = L.lxw_step(b, st, 0.0, 0.3, diag=True)
        assert d["status"] == 0
        skipped += d["n_mlp_skip"]
    Qb = L.to_q64(b, st)
    off = b.offsets
    for k in range(len(sizes)):
        assert torch.equal(Qb[off[k]:off[k + 1]], singles[k][0]), k
    assert skipped == sum(x[1] for x in singles) and skipped > 0


def test_batch_against_oracle_problem_by_problem(L):
    """Four problems of different sizes (one of 25 cells, less than a tile)
    and data in one batched mixed solver with persistent CTAs: each
    problem's slice against the oracle stepping that problem alone.
    (1) From a shared state, one step: averages within 1e-5 of the largest,
    modes within 1e-3 of their scale, relative L1 within 1e-5 (the FP32
    budget of one step), and each problem's own s and dt equal to the
    oracle's (s within the FP32 speed inflation 3e-5).  (2) From the initial
    data, 8 steps: relative L1 within 1e-4 per problem."""
    from oracle import oracle as O
    sizes = [5, 13, 24, 9]
    cfl = 0.3
    opt = L.lxw_options_default(precision=L.PREC_MIXED, ctas_per_sm=2)
    probs = [quadrant_problem(L, n, 400 + k) for k, n in enumerate(sizes)]
    b = L.lxw_batch_create([m for m, _ in probs], 2, opt, stream=torch.cuda.current_stream())
    Q = torch.cat([projected(L, L.lxw_solver_create(m, 2, stream=torch.cuda.current_stream()), ic)
                   for m, ic in probs])
    st = L.new_state(b, Q)
    Q0 = L.to_q64(b, st).cpu().numpy()                 # FP32 modes: the inputs both sides see
    off = b.offsets
    oracles = [O.Solver(O.Mesh.cartesian(n, n, (0.0, 1.0, 0.0, 1.0), (2, 2, 2, 2)), 2) for n in sizes]
    # (2) 8 steps from the initial data
    Qos = [Q0[off[k]:off[k + 1]].copy() for k in range(len(sizes))]
    for _ in range(8):
        L.lxw_step(b, st, 0.0, cfl)
        for so, Qo in zip(oracles, Qos):
            so.step(Qo, cfl=cfl)
    Qb = L.to_q64(b, st).cpu().numpy()
    for k, Qo in enumerate(Qos):
        Qg = Qb[off[k]:off[k + 1]]
        assert np.abs(Qg - Qo).sum() / np.abs(Qo).sum() < 1e-4, k
    # (1) one step from the shared state after those 8
    Qs = Qb.copy()
    Qs[:, :, 1:] = Qs[:, :, 1:].astype(np.float32)
    st = L.new_state(b, torch.from_numpy(Qs).cuda())
    d = L.lxw_step(b, st, 0.0, cfl, diag=True)
    assert d["status"] == 0
    sv, dv = L.lxw_batch_scalars(b)
    Qb = L.to_q64(b, st).cpu().numpy()
    for k, so in enumerate(oracles):
        Qo = Qs[off[k]:off[k + 1]].copy()
        do = so.step(Qo, cfl=cfl)
        Qg = Qb[off[k]:off[k + 1]]
        sc = np.abs(Qo).max(axis=0, keepdims=True) + 1e-3
        assert np.abs(Qg[:, :, 0] - Qo[:, :, 0]).max() < 1e-5 * np.abs(Qo[:, :, 0]).max(), k
        assert (np.abs(Qg - Qo) / sc).max() < 1e-3, k
        assert np.abs(Qg - Qo).sum() / np.abs(Qo).sum() < 1e-5, k
        assert abs(sv[k] / do["s"] - 1) < 3e-5, k
        assert abs(dv[k] / do["dt"] - 1) < 3e-5, k
    assert len(set(np.round(dv, 12))) == len(sizes)   # four different time steps
