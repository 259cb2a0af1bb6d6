"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances come from the arithmetic: both sides are FP64 with the same
operations in a different order (the GPU fuses multiply-adds), so one step
agrees to ~1e-15 relative; limiter parameters near vacuum (theta ~ 1e-12 from
the secant at a point pinned at rho = eps0) agree in absolute terms; the
spec bar is a relative L1 of 1e-11 after 100 steps of the smooth case.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QUAD, TRI = 0, 1
VARIANTS = [(QUAD, 2), (QUAD, 3), (TRI, 2), (TRI, 3)]


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1601_08145_gb300 import build
    build.build()
    from paper_1601_08145_gb300 import lxw
    return lxw


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.lib()
    return oracle


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def make_pair(L, O, kind, deg, n, bc=(0, 0, 0, 0), box=(0.0, 1.0, 0.0, 1.0), jitter=0.2, seed=20160129,
              shock=True, tri_bc=None, **opt):
    if kind == QUAD:
        om = O.Mesh.cartesian(n, n, box, bc)
        lm = L.lxw_mesh_cartesian(n, n, box, bc)
    else:
        xy, tv = synth.structured_triangles(n, jitter=jitter, seed=seed, box=box)
        ebc = None if tri_bc is None else np.full((len(tv), 3), tri_bc, dtype=np.int32)
        om = O.Mesh.triangles(xy, tv, ebc)
        lm = L.lxw_mesh_triangles(xy, tv, ebc)
    os_ = O.Solver(om, deg, shock_limiter=shock, **opt)
    o = L.lxw_options_default(shock_limiter=int(shock))
    for k, v in opt.items():
        setattr(o, k, v)
    ls = L.lxw_solver_create(lm, deg, o, stream=torch.cuda.current_stream())
    return os_, ls


def gpu(Q):
    return torch.from_numpy(np.ascontiguousarray(Q)).cuda()


def lib_project(L, ls, ic):
    xy = L.lxw_projection_points(ls)
    r, u, v, p = ic(xy[..., 0], xy[..., 1])
    prim = np.stack(np.broadcast_arrays(r, u, v, p), axis=-1)
    Q = torch.zeros(ls.state_shape, dtype=torch.float64, device="cuda")
    L.lxw_project(ls, gpu(prim), Q)
    torch.cuda.synchronize()
    return Q


@pytest.mark.parametrize("kind,deg", VARIANTS)
def test_projection_parity(L, O, kind, deg):
    os_, ls = make_pair(L, O, kind, deg, 7)
    assert np.allclose(L.lxw_projection_points(ls), os_.projection_points(), rtol=0, atol=1e-15)
    Qo = os_.project_fn(synth.ic_smooth)
    Qg = lib_project(L, ls, synth.ic_smooth).cpu().numpy()
    assert np.abs(Qg - Qo).max() < 1e-14


@pytest.mark.parametrize("kind,deg", VARIANTS)
def test_moment_limiter_and_speed_parity(L, O, kind, deg):
    os_, ls = make_pair(L, O, kind, deg, 9)
    Q0 = synth.random_modal_state(os_.N, os_.ML, seed=41 + deg, amp=1.2)
    Q0[::3, :, 1:] *= 0.05
    Qo = Q0.copy()
    tho, _ = os_.moment_limit(Qo)
    so = os_.wave_speed(Qo)
    Qg = gpu(Q0); thg = torch.zeros(os_.N, dtype=torch.float64, device="cuda")
    sg = torch.zeros(1, dtype=torch.float64, device="cuda")
    L.lxw_moment_limit(ls, Qg, thg, sg)
    torch.cuda.synchronize()
    assert np.abs(thg.cpu().numpy() - tho).max() < 1e-9
    assert np.array_equal(thg.cpu().numpy() == 1.0, tho == 1.0)
    assert np.abs(Qg.cpu().numpy() - Qo).max() < 1e-13 * np.abs(Q0).max()
    assert abs(sg.item() - so) <= 1e-14 * so


@pytest.mark.parametrize("kind,deg", VARIANTS)
def test_shock_limiter_parity(L, O, kind, deg):
    os_, ls = make_pair(L, O, kind, deg, 9, bc=(1, 1, 2, 2), tri_bc=1, alpha0=20.0)
    Q0 = synth.random_modal_state(os_.N, os_.ML, seed=7 + deg, amp=0.2)
    Qo = Q0.copy()
    tho = os_.shock_limit(Qo)
    Qg = gpu(Q0); thg = torch.zeros(os_.N, dtype=torch.float64, device="cuda")
    L.lxw_shock_limit(ls, Qg, thg)
    torch.cuda.synchronize()
    assert (tho < 1).sum() > 5
    assert np.abs(thg.cpu().numpy() - tho).max() < 1e-12
    assert np.abs(Qg.cpu().numpy() - Qo).max() < 1e-13 * np.abs(Q0).max()


def step_both(L, os_, ls, Q0, cfl, dt=0.0):
    Qo = Q0.copy()
    do = os_.step(Qo, dt=dt, cfl=cfl, want_theta=True)
    Qg = gpu(Q0)
    tc = torch.zeros((2, os_.N), dtype=torch.float64, device="cuda")
    te = torch.zeros((os_.N, os_.E), dtype=torch.float64, device="cuda")
    dg = L.lxw_step(ls, Qg, dt, cfl, diag=True, theta_cell=tc, theta_edge=te)
    torch.cuda.synchronize()
    return Qo, do, Qg.cpu().numpy(), dg, tc.cpu().numpy(), te.cpu().numpy()


@pytest.mark.parametrize("kind,deg", VARIANTS)
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_one_step_parity_limiters_active(L, O, kind, deg, bc):
    """One step from the same random state with every limiter exercised."""
    if kind == TRI and bc == 0:
        pytest.skip("triangle meshes have no periodic sides")
    os_, ls = make_pair(L, O, kind, deg, 12, bc=(bc,) * 4, tri_bc=bc if kind == TRI else None, alpha0=50.0)
    Q0 = synth.random_modal_state(os_.N, os_.ML, seed=100 + 10 * bc + deg, amp=0.3,
                                  rho_range=(0.01, 3.0), p_range=(0.001, 3.0))
    Qo, do, Qg, dg, tc, te = step_both(L, os_, ls, Q0, cfl=0.9)
    assert do["status"] == 0 and dg["status"] == 0
    # s is a max over point values of states limited near vacuum: agreement to 1e-13
    assert abs(dg["s"] - do["s"]) <= 1e-13 * do["s"] and abs(dg["dt"] - do["dt"]) <= 1e-13 * do["dt"]
    assert do["n_mom"] > 0 and do["n_sc"] > 0
    assert rel_l1(Qg, Qo) < 1e-13
    assert np.abs(Qg - Qo).max() < 1e-11 * np.abs(Qo).max()
    assert np.abs(tc[0] - do["theta_mom"]).max() < 1e-9
    assert np.abs(tc[1] - do["theta_sc"]).max() < 1e-9
    assert np.abs(te - do["theta_edge"]).max() < 1e-9
    assert (dg["n_mom"], dg["n_edge"], dg["n_sc"]) == (do["n_mom"], do["n_edge"], do["n_sc"])
    for k in ("mass", "momx", "momy", "energy"):
        assert abs(dg[k] - do[k]) <= 1e-12 * max(1.0, abs(do[k]))
    assert abs(dg["min_rho"] - do["min_rho"]) <= 1e-13 * abs(do["min_rho"])


def run_both(L, os_, ls, Qo, Qg, nsteps, cfl):
    for _ in range(nsteps):
        os_.step(Qo, cfl=cfl)
    L.lxw_run(ls, Qg, nsteps, cfl)
    torch.cuda.synchronize()
    return Qo, Qg.cpu().numpy()


def test_smooth_wave_100_steps_to_1e11(L, O):
    """32x32 periodic P2 smooth wave, CFL 0.1, all limiters on: relative L1
    of the GPU FP64 state against the oracle after 100 steps."""
    os_, ls = make_pair(L, O, QUAD, 2, 32)
    Qo = os_.project_fn(synth.ic_smooth)
    Qg = lib_project(L, ls, synth.ic_smooth)
    Qo, Qgn = run_both(L, os_, ls, Qo, Qg, 100, 0.1)
    err = rel_l1(Qgn, Qo)
    print(f"smooth 100 steps relative L1 {err:.3e}")
    assert err < 1e-11


def oracle_sensitivity(O, om, deg, Q0, nsteps, cfl):
    """Relative L1 by which the oracle's own state moves after nsteps when
    its input is perturbed by 1e-15 (relative, seeded): the round-off
    amplification of the limiters' discontinuous decisions on this problem.
    A GPU that rounds differently cannot be held closer than this."""
    a, b = O.Solver(om, deg), O.Solver(om, deg)
    Q1 = Q0.copy()
    Q2 = Q0 * (1.0 + 1e-15 * np.random.default_rng(1).standard_normal(Q0.shape))
    for _ in range(nsteps):
        a.step(Q1, cfl=cfl); b.step(Q2, cfl=cfl)
    return rel_l1(Q2, Q1)


@pytest.mark.parametrize("deg", [2, 3])
def test_blast_and_rarefaction_multi_step(L, O, deg):
    """40 steps with the limiters active (blast: walls; rarefaction: jittered
    triangles): relative L1 within 1e-11, or within 10x the oracle's own
    round-off amplification on the problem where that is larger (measured
    1.3e-11 for the P3 rarefaction: a limiter decision flips between steps
    20 and 40 under a 1e-15 perturbation)."""
    os_, ls = make_pair(L, O, QUAD, deg, 32, bc=(1, 1, 1, 1), box=(-1.1, 1.1, -1.1, 1.1))
    Qo = os_.project_fn(synth.ic_blast(32))
    Qg = lib_project(L, ls, synth.ic_blast(32))
    Qo, Qgn = run_both(L, os_, ls, Qo, Qg, 40, 0.1)
    assert rel_l1(Qgn, Qo) < 1e-11
    os_, ls = make_pair(L, O, TRI, deg, 16)
    Qo = os_.project_fn(synth.ic_rarefy)
    sens = oracle_sensitivity(O, os_.mesh, deg, Qo, 40, 0.1)
    Qg = lib_project(L, ls, synth.ic_rarefy)
    Qo, Qgn = run_both(L, os_, ls, Qo, Qg, 40, 0.1)
    err = rel_l1(Qgn, Qo)
    print(f"rarefaction P{deg}: GPU vs oracle {err:.2e}, oracle self-sensitivity {sens:.2e}")
    assert err < max(1e-11, 10.0 * sens)


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 5), (13, 11), (3, 2)])
def test_edge_case_meshes(L, O, nx, ny):
    """Self-neighbours (1x1 periodic), a one-cell-wide strip, a ragged tail
    (143 elements: not a multiple of the CTA size), a tiny mesh."""
    om = O.Mesh.cartesian(nx, ny); os_ = O.Solver(om, 2)
    lm = L.lxw_mesh_cartesian(nx, ny); ls = L.lxw_solver_create(lm, 2, stream=torch.cuda.current_stream())
    Q0 = synth.random_modal_state(nx * ny, 6, seed=nx * 100 + ny, amp=0.3)
    Qo, do, Qg, dg, tc, te = step_both(L, os_, ls, Q0, cfl=0.5)
    assert rel_l1(Qg, Qo) < 1e-13
    assert np.abs(te - do["theta_edge"]).max() < 1e-9


def test_two_triangles(L, O):
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=float)
    tv = np.array([[0, 1, 2], [0, 2, 3]])
    for bc in (1, 2):
        ebc = np.full((2, 3), bc, dtype=np.int32)
        os_ = O.Solver(O.Mesh.triangles(xy, tv, ebc), 2)
        ls = L.lxw_solver_create(L.lxw_mesh_triangles(xy, tv, ebc), 2, stream=torch.cuda.current_stream())
        Q0 = synth.random_modal_state(2, 6, seed=5 + bc, amp=0.2)
        Qo, do, Qg, dg, tc, te = step_both(L, os_, ls, Q0, cfl=0.5)
        assert rel_l1(Qg, Qo) < 1e-13


def test_graph_replay_matches_single_steps(L, O):
    os_, ls = make_pair(L, O, TRI, 2, 10)
    Q0 = os_.project_fn(synth.ic_rarefy)
    A = gpu(Q0); B = gpu(Q0)
    for _ in range(7):
        L.lxw_step(ls, A, 0.0, 0.2)
    L.lxw_run(ls, B, 7, 0.2)
    torch.cuda.synchronize()
    assert torch.equal(A, B)
    # host-buffer path: same result as the device path
    H = Q0.copy()
    L.lxw_run_host(ls, H, 7, 0.2)
    assert np.array_equal(H, A.cpu().numpy())


def test_diagnostics_conservation_and_status(L, O):
    os_, ls = make_pair(L, O, QUAD, 2, 16)
    Q = gpu(synth.random_modal_state(os_.N, os_.ML, seed=3, amp=0.05))
    d0 = L.lxw_step(ls, Q, 0.0, 0.1, diag=True)
    for _ in range(20):
        d = L.lxw_step(ls, Q, 0.0, 0.1, diag=True)
    for k in ("mass", "momx", "momy", "energy"):
        assert abs(d[k] - d0[k]) < 1e-13 * max(1.0, abs(d0[k]))
    assert d["status"] == 0 and d["return_status"] == L.OK
    # a non-positive average is reported, not hidden
    Qb = synth.random_modal_state(os_.N, os_.ML, seed=4, amp=0.05)
    Qb[5, 0, 0] = -1.0
    d = L.lxw_step(ls, gpu(Qb), 0.0, 0.1, diag=True)
    assert d["status"] & L.ST_NONPOSITIVE and d["return_status"] == L.ERR_NONPOSITIVE
    assert L.lxw_step_launches(ls) == 6


def test_full_size_rarefaction_one_step(L, O):
    """The benchmarked workload (224x224x2 jittered triangles, P2, the launch
    configuration the benchmark times) from a random state with every limiter
    active: every output element against the oracle."""
    os_, ls = make_pair(L, O, TRI, 2, 224)
    Q0 = synth.random_modal_state(os_.N, os_.ML, seed=2024, amp=0.3, rho_range=(0.01, 3.0), p_range=(0.001, 3.0))
    Qo, do, Qg, dg, tc, te = step_both(L, os_, ls, Q0, cfl=0.9)
    assert rel_l1(Qg, Qo) < 1e-13
    assert np.abs(te - do["theta_edge"]).max() < 1e-9
    assert np.abs(tc[0] - do["theta_mom"]).max() < 1e-9
    Qo = os_.project_fn(synth.ic_rarefy)
    Qg = lib_project(L, ls, synth.ic_rarefy)
    Qo, Qgn = run_both(L, os_, ls, Qo, Qg, 3, 0.1)
    assert rel_l1(Qgn, Qo) < 1e-13


def test_full_size_blast_step_and_limiter_counts(L, O):
    """The 1024^2 blast (reflective walls, P2): after 20 oracle steps from the
    point-energy data, one FP64 step of both sides from that shared state (the
    moment and shock limiters active at the front) agrees element by element,
    with the same limiter-activity counts."""
    n = 1024
    box = (-1.1, 1.1, -1.1, 1.1)
    os_, ls = make_pair(L, O, QUAD, 2, n, bc=(1, 1, 1, 1), box=box)
    Q0 = os_.project_fn(synth.ic_blast(n))
    for _ in range(20):
        os_.step(Q0, cfl=0.1)
    Qo, do, Qg, dg, tc, te = step_both(L, os_, ls, Q0, cfl=0.1)
    assert dg["status"] == 0 and do["status"] == 0 and dg["min_p"] > 0
    assert rel_l1(Qg, Qo) < 1e-12
    assert do["n_mom"] > 0 and do["n_sc"] > 0
    for k in ("n_mom", "n_edge", "n_sc"):
        assert dg[k] == do[k], (k, dg[k], do[k])
    assert np.abs(tc[0] - do["theta_mom"]).max() < 1e-9 and np.abs(tc[1] - do["theta_sc"]).max() < 1e-9


@pytest.mark.parametrize("mixed", [False, True])
def test_blast_keeps_its_fourfold_symmetry(L, mixed):
    """64^2 blast, 150 steps: density and energy averages symmetric under
    x -> -x, y -> -y and x <-> y.  Mirrored cells add their edge fluxes in a
    different local order, so the two halves differ by rounding, which the
    limiters' discontinuous decisions amplify over the steps at the front:
    FP64 within 5e-9 of the largest value (measured 1.7e-9), mixed (FP32
    bulk) within 1e-2 (measured 1.8e-3) -- a wrong sign in a wall or a
    mirrored table would break it at O(1)."""
    n = 64
    mesh = L.lxw_mesh_cartesian(n, n, (-1.1, 1.1, -1.1, 1.1), (1, 1, 1, 1))
    o = L.lxw_options_default(precision=L.PREC_MIXED if mixed else L.PREC_FP64)
    s = L.lxw_solver_create(mesh, 2, o, stream=torch.cuda.current_stream())
    Q = lib_project(L, s, synth.ic_blast(n)) if not mixed else None
    if mixed:
        s64 = L.lxw_solver_create(mesh, 2, stream=torch.cuda.current_stream())
        Q = L.new_state(s, lib_project(L, s64, synth.ic_blast(n)))
    for _ in range(150):
        d = L.lxw_step(s, Q, 0.0, 0.1, diag=True)
        assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0
    Qh = (L.to_q64(s, Q) if mixed else Q).cpu().numpy()
    tol = 1e-2 if mixed else 5e-9
    worst = 0.0
    for v in (0, 3):
        A = Qh[:, v, 0].reshape(n, n)
        sc = np.abs(A).max()
        for B in (A[:, ::-1], A[::-1, :], A.T):
            worst = max(worst, np.abs(A - B).max() / sc)
    print(f"blast symmetry ({'mixed' if mixed else 'fp64'}): {worst:.2e}")
    assert worst < tol


@pytest.mark.parametrize("mixed", [False, True])
def test_double_rarefaction_1d_as_y_invariant_2d(L, O, mixed):
    """The paper's 1D double rarefaction (rho 7, u -+1, p 0.2; Sec. 4.1) on
    a 128 x 4 strip, periodic in y and transparent in x: positive at every
    step, the y-carrying modes stay zero (y-invariance), and the result
    matches the oracle's (FP64 1e-12; mixed within the FP32 budget)."""
    nx, ny = 128, 4
    bc = (2, 2, 0, 0)          # left, right transparent; bottom, top periodic
    ic = lambda x, y: (7.0 + 0 * x, np.where(x < 0.5, -1.0, 1.0), 0 * x, 0.2 + 0 * x)
    om = O.Mesh.cartesian(nx, ny, (0.0, 1.0, 0.0, 1.0), bc)
    so = O.Solver(om, 2)
    Qo = so.project_fn(ic)
    lm = L.lxw_mesh_cartesian(nx, ny, (0.0, 1.0, 0.0, 1.0), bc)
    o = L.lxw_options_default(precision=L.PREC_MIXED if mixed else L.PREC_FP64)
    s = L.lxw_solver_create(lm, 2, o, stream=torch.cuda.current_stream())
    s64 = L.lxw_solver_create(lm, 2, stream=torch.cuda.current_stream())
    Q64 = lib_project(L, s64, ic)
    Qg = L.new_state(s, Q64) if mixed else Q64
    if mixed:
        Qo[:, :, 1:] = L.to_q64(s, Qg).cpu().numpy()[:, :, 1:]      # both start from FP32 modes
    for _ in range(200):
        do = so.step(Qo, cfl=0.1)
        d = L.lxw_step(s, Qg, 0.0, 0.1, diag=True)
        assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0
        assert do["min_rho"] > 0 and do["min_p"] > 0
    Qh = (L.to_q64(s, Qg) if mixed else Qg).cpu().numpy()
    # y-invariance: modes carrying eta (L1(y), L1(x)L1(y), L2(y)) and the y-momentum vanish, to
    # round-off (FP64) or to the FP32 rounding of the modal sums relative to each variable's scale
    scale = np.abs(Qh[:, :, 0]).max(axis=0)
    scale[1] = scale[2] = max(scale[1], scale[2])        # both momenta on the momentum scale
    tol = (1e-5 if mixed else 1e-14) * scale
    for v in range(4):
        assert np.abs(Qh[:, v, [2, 3, 5]]).max() < tol[v], v
    assert np.abs(Qh[:, 2, :]).max() < tol.max()
    err = rel_l1(Qh, Qo)
    print(f"double rarefaction ({'mixed' if mixed else 'fp64'}): relative L1 vs oracle {err:.2e}")
    assert err < (1e-4 if mixed else 1e-12)


@pytest.mark.parametrize("kind", [QUAD, TRI])
def test_fourth_order_ck_matches_oracle(L, O, kind):
    """ck_order 4 (dt^3/24 F_ttt added to the time-averaged flux) on P3: 20
    steps of the smooth wave against the oracle with the same option, as
    close as the third-order runs are (1e-12 relative L1, or 10x the
    third-order distance where the two sides' P3 tables differ more); the
    added term is active (it moves the state by more than round-off)."""
    err, states = {}, {}
    for order in (3, 4):
        os_, ls = make_pair(L, O, kind, 3, 12, ck_order=order)
        Qo = os_.project_fn(synth.ic_smooth)
        Qg = lib_project(L, ls, synth.ic_smooth)
        Qo, Qgn = run_both(L, os_, ls, Qo, Qg, 20, 0.1)
        err[order] = rel_l1(Qgn, Qo)
        states[order] = Qgn
    print(f"P3 {'quad' if kind == QUAD else 'tri'}: GPU vs oracle, CK order 3 {err[3]:.2e}, order 4 {err[4]:.2e}")
    assert err[4] < max(1e-12, 10.0 * err[3])
    d = rel_l1(states[3], states[4])
    assert 1e-11 < d < 1e-5, d
