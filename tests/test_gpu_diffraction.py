"""The shock-diffraction setting of Sec. 4 on the GPU: masked Cartesian
meshes (the step), the inflow boundary, against the oracle.

Tolerances: the FP64 form repeats the oracle's operations in another order
(fused multiply-adds), ~1e-15 relative per step, which the limiters at the
Mach 5.09 shock can amplify by a few orders over tens of steps; the mixed
form carries FP32 fluxes (~1e-7 relative per step in the averages)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_, R_, INFLOW = 2, 1, 3
G = 1.4


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


POST = synth.normal_shock_state(synth.DIFFRACTION_MACH)


def conserved(prim):
    r, u, v, p = prim
    return np.array([r, r * u, r * v, p / (G - 1.0) + 0.5 * r * (u * u + v * v)])


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def gpu_solver(L, mesh, deg, mixed, **opt):
    o = L.lxw_options_default(precision=L.PREC_MIXED if mixed else L.PREC_FP64)
    for k, v in opt.items():
        setattr(o, k, v)
    s = L.lxw_solver_create(mesh, deg, o, stream=torch.cuda.current_stream())
    return s


def gpu_state(L, s, Q):
    Q64 = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    return L.new_state(s, Q64) if s.mixed else Q64


def gpu_q64(L, s, st):
    return (L.to_q64(s, st) if s.mixed else st).cpu().numpy()


def diffraction(L, O, nx, ny, deg, mixed, **opt):
    mask = synth.diffraction_mask(nx, ny)
    bc = synth.DIFFRACTION_BC
    so = O.Solver(O.Mesh.cartesian_masked(nx, ny, synth.DIFFRACTION_BOX, bc, mask, R_), deg, **opt)
    so.set_inflow(POST)
    s = gpu_solver(L, L.lxw_mesh_cartesian_masked(nx, ny, synth.DIFFRACTION_BOX, bc, mask, L.BC_REFLECT),
                   deg, mixed, **opt)
    L.lxw_solver_set_inflow(s, POST)
    assert s.N == so.N == int(mask.sum())
    return so, s


def test_masked_mesh_and_inflow_argument_errors(L):
    mask = np.ones((3, 4), np.uint8)
    with pytest.raises(L.LxwError) as e:
        L.lxw_mesh_cartesian_masked(4, 3, (0, 1, 0, 1), (2, 2, 2, 2), mask, mask_bc=0)   # periodic mask faces
    assert e.value.code == L.ERR_ARG
    with pytest.raises(L.LxwError) as e:
        L.lxw_mesh_cartesian_masked(4, 3, (0, 1, 0, 1), (2, 2, 2, 2), 0 * mask)           # no cell kept
    assert e.value.code == L.ERR_ARG
    m = L.lxw_mesh_cartesian_masked(4, 3, (0, 1, 0, 1), (2, 2, 2, 2), mask)
    s = gpu_solver(L, m, 2, False)
    with pytest.raises(L.LxwError) as e:
        L.lxw_solver_set_inflow(s, (1.0, 0.0, 0.0, -1.0))
    assert e.value.code == L.ERR_ARG


@pytest.mark.parametrize("mixed", [False, True], ids=["fp64", "mixed"])
@pytest.mark.parametrize("deg", [2, 3])
def test_diffraction_parity_with_oracle(L, O, deg, mixed):
    """The step at 1/10 of the paper's resolution (39 x 33 cells less the
    step), 40 steps at CFL 0.1 with every limiter on: positive at every step
    and the state matches the oracle's."""
    so, s = diffraction(L, O, 39, 33, deg, mixed)
    Qo = so.project_fn(synth.ic_diffraction)
    if mixed:
        Qo[:, :, 1:] = Qo[:, :, 1:].astype(np.float32)
    st = gpu_state(L, s, Qo)
    lim = 0
    for k in range(40):
        do = so.step(Qo, cfl=0.1)
        d = L.lxw_step(s, st, 0.0, 0.1, diag=True)
        assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0, (k, d)
        assert do["status"] == 0
        assert abs(d["dt"] / do["dt"] - 1) < (3e-5 if mixed else 1e-13)
        lim += d["n_mom"] + d["n_edge"] + d["n_sc"]
    Qg = gpu_q64(L, s, st)
    err = rel_l1(Qg, Qo)
    print(f"diffraction P{deg} ({'mixed' if mixed else 'fp64'}): relative L1 vs oracle {err:.2e}, limited {lim}")
    assert lim > 0
    assert err < (2e-4 if mixed else 1e-10)


@pytest.mark.parametrize("mixed", [False, True], ids=["fp64", "mixed"])
def test_inflow_driven_shock_closed_form(L, mixed):
    """Mach 5.09 shock driven by the inflow along a 96 x 2 channel (the
    oracle's pin): the integrals of mass, momentum and energy change by
    exactly the inflow minus outflow fluxes, the shock sits at x_s + 5.09 t."""
    q1, q0 = conserved(POST), conserved((1.4, 0.0, 0.0, 1.0))
    nx, Lx, H, xs = 96, 3.0, 0.0625, 1.25
    s = gpu_solver(L, L.lxw_mesh_cartesian(nx, 2, (0.0, Lx, 0.0, H), (INFLOW, T_, R_, R_)), 2, mixed)
    L.lxw_solver_set_inflow(s, POST)
    cx = (np.arange(nx) + 0.5) * Lx / nx
    Q = np.zeros((2 * nx, 4, 6))
    Q[:, :, 0] = np.where((np.tile(cx, 2) < xs)[:, None], q1[None, :], q0[None, :])
    a = (Lx / nx) * (H / 2)
    tot0 = a * Q[:, :, 0].sum(axis=0)
    st = gpu_state(L, s, Q)
    n, dt = 400, 2e-4
    for k in range(n):
        d = L.lxw_step(s, st, dt, 0.0, diag=(k % 50 == 49))
        if d is not None:
            assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0, (k, d)
    Qg = gpu_q64(L, s, st)
    tot = a * Qg[:, :, 0].sum(axis=0)
    t = n * dt
    F1 = np.array([q1[1], q1[1] * POST[1] + POST[3], 0.0, POST[1] * (q1[3] + POST[3])])
    F0 = np.array([0.0, 1.0, 0.0, 0.0])
    expect = tot0 + (F1 - F0) * H * t
    tol = 1e-6 if mixed else 1e-13
    for v in (0, 1, 3):
        assert abs(tot[v] - expect[v]) <= tol * abs(expect[v]), (v, tot[v], expect[v])
    rho = Qg[:nx, 0, 0]
    mid = 0.5 * (POST[0] + 1.4)
    k = int(np.argmax(rho < mid))
    x_half = cx[k - 1] + (cx[k] - cx[k - 1]) * (mid - rho[k - 1]) / (rho[k] - rho[k - 1])
    assert abs(x_half - (xs + 5.09 * t)) < 1.5 * Lx / nx


@pytest.mark.parametrize("mixed", [False, True], ids=["fp64", "mixed"])
def test_inflow_side_on_triangles(L, O, mixed):
    """Jittered triangles of the unit square, inflow on the left side (edge
    codes), walls below and above, transparent on the right: 30 steps against
    the oracle."""
    xy, tv = synth.structured_triangles(16, jitter=0.2, seed=20160129)
    ebc = np.full((len(tv), 3), T_, dtype=np.int32)
    for e in range(len(tv)):
        for k in range(3):
            a, b = xy[tv[e, k]], xy[tv[e, (k + 1) % 3]]
            mx, my = 0.5 * (a + b)
            if mx < 1e-12:
                ebc[e, k] = INFLOW
            elif my < 1e-12 or my > 1 - 1e-12:
                ebc[e, k] = R_
    prim_in = (2.5, 1.2, 0.1, 2.0)
    so = O.Solver(O.Mesh.triangles(xy, tv, ebc), 2)
    so.set_inflow(prim_in)
    s = gpu_solver(L, L.lxw_mesh_triangles(xy, tv, ebc), 2, mixed)
    L.lxw_solver_set_inflow(s, prim_in)

    def ic(x, y):
        return (1.0 + 0.2 * np.sin(6 * y) + 0 * x, 0.3 + 0 * x, 0 * x, np.where(x < 0.5, 1.0, 0.4))

    Qo = so.project_fn(ic)
    if mixed:
        Qo[:, :, 1:] = Qo[:, :, 1:].astype(np.float32)
    st = gpu_state(L, s, Qo)
    for k in range(30):
        so.step(Qo, cfl=0.1)
        d = L.lxw_step(s, st, 0.0, 0.1, diag=True)
        assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0, (k, d)
    err = rel_l1(gpu_q64(L, s, st), Qo)
    print(f"triangles with inflow ({'mixed' if mixed else 'fp64'}): relative L1 vs oracle {err:.2e}")
    assert err < (1e-4 if mixed else 1e-11)


def test_mixed_shock_limiter_and_features_next_to_the_inflow(L, O):
    """The mixed form's shock limiter and gate features read the inflow state
    as the neighbour average of the inflow cells: against the oracle on the
    state the limiter saw (FP32 averages)."""
    nx, ny = 39, 33
    so, s = diffraction(L, O, nx, ny, 2, True, alpha0=50.0)
    s0 = gpu_solver(L, L.lxw_mesh_cartesian_masked(nx, ny, synth.DIFFRACTION_BOX, synth.DIFFRACTION_BC,
                                                   synth.diffraction_mask(nx, ny), L.BC_REFLECT),
                    2, True, alpha0=50.0, shock_limiter=0)
    L.lxw_solver_set_inflow(s0, POST)
    Q0 = so.project_fn(synth.ic_diffraction)
    # perturb the first columns so that the inflow cells are limited against q_in
    rng = np.random.default_rng(5)
    a, _, cx, cy = so.mesh.geometry()
    near = cx < 1.5
    Q0[near, :, 1:] += 0.05 * rng.standard_normal((near.sum(), 4, 5)) * np.abs(Q0[near, :, :1])
    Q0[:, :, 1:] = Q0[:, :, 1:].astype(np.float32)
    st = gpu_state(L, s, Q0)
    A = st.clone(); B = st.clone()
    F, th = L.lxw_step_dump(s, A, 0.1)
    L.lxw_step(s0, B, 0.0, 0.1)
    Qpre = L.to_q64(s0, B).cpu().numpy()
    Qpre[:, :, 0] = Qpre[:, :, 0].astype(np.float32)
    Fo = so.features(Qpre)
    Fg = F.double().cpu().numpy()
    assert np.abs(Fg - Fo).max() < 1e-5 * (1 + np.abs(Fo).max())
    tho = so.shock_limit(Qpre.copy())
    thg = th.cpu().numpy()
    first = np.where(cx < 1.0 / 3.0)[0]
    assert (tho[first] < 1).sum() > 3
    assert np.abs(thg - tho).max() < 1e-3
    assert np.mean(np.abs(thg - tho) < 1e-5) > 0.99
