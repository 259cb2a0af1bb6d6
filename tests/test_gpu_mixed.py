"""The mixed-precision form (FP32 bulk, FP64 averages / update / limiter
solves) against the FP64 oracle and the FP64 GPU form.

Tolerances follow from the arithmetic: one mixed step differs from the FP64
step by FP32 rounding of the bulk terms (~1e-6 relative in the higher modes,
~1e-7 of the flux increment in the averages); conservation stays at FP64
round-off because both sides of an edge add the same FP32 flux, negated, in
FP64; positivity of the averages is kept exactly by the FP64 limiter.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QUAD, TRI = 0, 1


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


def solver(L, kind, deg, n, mixed=True, bc=(0, 0, 0, 0), box=(0.0, 1.0, 0.0, 1.0), tri_bc=None, **opt):
    if kind == QUAD:
        mesh = L.lxw_mesh_cartesian(n, n, box, bc)
    else:
        xy, tv = synth.structured_triangles(n, jitter=0.2, seed=20160129, box=box)
        ebc = None if tri_bc is None else np.full((len(tv), 3), tri_bc, dtype=np.int32)
        mesh = L.lxw_mesh_triangles(xy, tv, ebc)
    o = L.lxw_options_default(precision=L.PREC_MIXED if mixed else L.PREC_FP64)
    for k, v in opt.items():
        setattr(o, k, v)
    return L.lxw_solver_create(mesh, deg, o, stream=torch.cuda.current_stream())


def oracle_solver(O, kind, deg, n, bc=(0, 0, 0, 0), box=(0.0, 1.0, 0.0, 1.0), tri_bc=None, **kw):
    if kind == QUAD:
        m = O.Mesh.cartesian(n, n, box, bc)
    else:
        xy, tv = synth.structured_triangles(n, jitter=0.2, seed=20160129, box=box)
        ebc = None if tri_bc is None else np.full((len(tv), 3), tri_bc, dtype=np.int32)
        m = O.Mesh.triangles(xy, tv, ebc)
    return O.Solver(m, deg, **kw)


def project(L, s, ic):
    xy = L.lxw_projection_points(s)
    r, u, v, p = ic(xy[..., 0], xy[..., 1])
    prim = torch.from_numpy(np.stack(np.broadcast_arrays(r, u, v, p), axis=-1).copy()).cuda()
    Q = torch.zeros(s.q64_shape, dtype=torch.float64, device="cuda")
    L.lxw_project(s, prim, Q)
    return Q


@pytest.mark.parametrize("kind,deg", [(QUAD, 2), (TRI, 3)])
def test_pack_roundtrip(L, kind, deg):
    s = solver(L, kind, deg, 9)
    Q0 = torch.from_numpy(synth.random_modal_state(s.N, s.ML, seed=3, amp=0.3)).cuda()
    st = L.new_state(s, Q0)
    Q1 = L.to_q64(s, st)
    torch.cuda.synchronize()
    assert torch.equal(Q1[:, :, 0], Q0[:, :, 0])                     # averages stay FP64
    assert torch.equal(Q1[:, :, 1:], Q0[:, :, 1:].float().double())  # higher modes are FP32
    # a source 8 bytes off a 16-byte boundary takes the scalar copy path: same state
    flat = torch.empty(Q0.numel() + 1, dtype=torch.float64, device="cuda")
    Qm = flat[1:].view(Q0.shape)
    Qm.copy_(Q0)
    assert Qm.data_ptr() % 16 == 8
    assert torch.equal(L.new_state(s, Qm), st)


@pytest.mark.parametrize("kind,deg", [(QUAD, 2), (QUAD, 3), (TRI, 2), (TRI, 3)])
def test_one_mixed_step_close_to_oracle(L, O, kind, deg):
    bc = 2
    s = solver(L, kind, deg, 12, bc=(bc,) * 4, tri_bc=bc if kind == TRI else None)
    so = oracle_solver(O, kind, deg, 12, bc=(bc,) * 4, tri_bc=bc if kind == TRI else None)
    Q0 = synth.random_modal_state(s.N, s.ML, seed=5 + deg, amp=0.3)
    Q0[:, :, 1:] = Q0[:, :, 1:].astype(np.float32)                    # both start from FP32-representable modes
    Qo = Q0.copy(); do = so.step(Qo, cfl=0.3)
    st = L.new_state(s, torch.from_numpy(Q0).cuda())
    d = L.lxw_step(s, st, 0.0, 0.3, diag=True)
    Qg = L.to_q64(s, st).cpu().numpy()
    assert d["status"] == 0 and do["status"] == 0
    assert abs(d["s"] / do["s"] - 1) < 3e-5
    sc = np.abs(Qo).max(axis=0, keepdims=True) + 1e-3
    assert np.abs(Qg[:, :, 0] - Qo[:, :, 0]).max() < 1e-5 * np.abs(Qo[:, :, 0]).max()
    assert (np.abs(Qg - Qo) / sc).max() < 1e-3
    assert np.abs(Qg - Qo).sum() / np.abs(Qo).sum() < 1e-5


def test_mixed_conservation_and_no_fallback_on_smooth_data(L):
    s = solver(L, QUAD, 2, 32)
    st = L.new_state(s, project(L, s, synth.ic_smooth))
    d0 = L.lxw_step(s, st, 0.0, 0.1, diag=True)
    for _ in range(30):
        d = L.lxw_step(s, st, 0.0, 0.1, diag=True)
        assert d["n_fp64_moment"] == 0 and d["n_fp64_edge"] == 0 and d["n_mom"] == 0 and d["n_edge"] == 0
    for k in ("mass", "momx", "momy", "energy"):
        assert abs(d[k] - d0[k]) <= 1e-13 * max(1.0, abs(d0[k]))


def test_mixed_positivity_blast_and_rarefaction(L):
    cases = [(QUAD, 2, 48, (1, 1, 1, 1), (-1.1, 1.1, -1.1, 1.1), synth.ic_blast(48), None),
             (TRI, 2, 24, (0, 0, 0, 0), (0.0, 1.0, 0.0, 1.0), synth.ic_rarefy, None),
             (TRI, 3, 16, (0, 0, 0, 0), (0.0, 1.0, 0.0, 1.0), synth.ic_rarefy, None)]
    for kind, deg, n, bc, box, ic, tb in cases:
        s = solver(L, kind, deg, n, bc=bc, box=box)
        st = L.new_state(s, project(L, s, ic))
        fb = 0
        for k in range(120):
            d = L.lxw_step(s, st, 0.0, 0.1, diag=True)
            assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0, (kind, deg, k, d)
            fb += d["n_fp64_moment"] + d["n_fp64_edge"]
        assert fb < 0.5 * 120 * s.N                     # the FP32 screens decide most cells


def test_mixed_l1_error_equals_fp64_on_exact_wave(L):
    """The smooth advected wave (32x32, P2, CFL 0.1, all limiters on) run to
    t = 0.1 exactly (lxw_run_to): the L1 error of the cell-average density
    against the exact cell averages, the norm the metric's "equal L1 error"
    names, is within 5 % of the FP64 GPU form's for the mixed form; the L2
    error of the DG density within 1 %."""
    from oracle import oracle as O   # only to project the exact solution and evaluate fields
    T = 0.1
    so = O.Solver(O.Mesh.cartesian(32, 32), 2)
    Qx = so.project_fn(lambda x, y: (synth.exact_smooth_density(x, y, T), 1.0 + 0 * x, 1.0 + 0 * x, 1.0 + 0 * x))
    xy = so.projection_points(); w = so.projection_weights()
    ex = synth.exact_smooth_density(xy[..., 0], xy[..., 1], T)
    l1, l2 = {}, {}
    for mixed in (False, True):
        s = solver(L, QUAD, 2, 32, mixed=mixed)
        Q = project(L, s, synth.ic_smooth)
        st = L.new_state(s, Q) if mixed else Q
        steps, t, _ = L.lxw_run_to(s, st, T, 0.1)
        assert t == T
        Qe = L.to_q64(s, st).cpu().numpy()
        l1[mixed] = float(np.mean(np.abs(Qe[:, 0, 0] - Qx[:, 0, 0])))
        q = so.eval_projection_points(Qe)[..., 0]
        l2[mixed] = float(np.sqrt(np.sum(w[None, :] * (q - ex) ** 2) / (32 * 32)))
    print("cell-average L1 errors fp64 / mixed", l1, "L2", l2)
    assert l1[True] <= 1.05 * l1[False]
    assert l2[True] <= 1.01 * l2[False]


def test_mixed_run_graph_and_host_path(L):
    s = solver(L, TRI, 2, 20)
    Q = project(L, s, synth.ic_rarefy)
    A = L.new_state(s, Q); B = L.new_state(s, Q)
    for _ in range(5):
        L.lxw_step(s, A, 0.0, 0.1)
    L.lxw_run(s, B, 5, 0.1)
    torch.cuda.synchronize()
    assert torch.equal(A, B)
    H = Q.cpu().numpy().copy()
    L.lxw_run_host(s, H, 5, 0.1)                        # pageable: staged copies
    assert np.array_equal(H, L.to_q64(s, A).cpu().numpy())
    P = Q.cpu().pin_memory()
    L.lxw_run_host(s, P, 5, 0.1)                        # pinned: read and written in place by the kernels
    assert np.array_equal(P.numpy(), H)
    # the solver's own layout on the host: DMA of the packed state both ways
    S = L.new_state(s, Q).cpu().pin_memory()
    L.lxw_run_host_state(s, S, 5, 0.1)
    assert torch.equal(S, A.cpu())
    # an FP64 solver's layout is Q[N][4][ML]
    s64 = solver(L, TRI, 2, 20, mixed=False)
    A64 = Q.clone(); L.lxw_run(s64, A64, 5, 0.1)
    S64 = Q.cpu().pin_memory()
    L.lxw_run_host_state(s64, S64, 5, 0.1)
    assert torch.equal(S64, A64.cpu())


def test_status_is_kept_until_a_diagnostic_step_reads_it(L):
    """Steps without diagnostics launch no reset: a non-positive average met
    by such a step is reported by the next step that asks for diagnostics,
    and cleared once reported."""
    s = solver(L, QUAD, 2, 12)
    Qb = synth.random_modal_state(s.N, s.ML, seed=4, amp=0.05)
    Qb[5, 0, 0] = -1.0
    L.lxw_step(s, L.new_state(s, torch.from_numpy(Qb).cuda()), 0.0, 0.1)      # no diagnostics
    good = L.new_state(s, torch.from_numpy(synth.random_modal_state(s.N, s.ML, seed=5, amp=0.05)).cuda())
    d = L.lxw_step(s, good, 0.0, 0.1, diag=True)
    assert d["status"] & L.ST_NONPOSITIVE and d["return_status"] == L.ERR_NONPOSITIVE
    d = L.lxw_step(s, good, 0.0, 0.1, diag=True)
    assert d["status"] == 0 and d["return_status"] == L.OK
    assert L.lxw_step_launches(s) == 5 and L.lxw_profile_phases(s) == 5


@pytest.mark.parametrize("kind,n,deg", [(TRI, 224, 2), (TRI, 224, 3), (QUAD, 1024, 2), (QUAD, 2048, 2)])
def test_full_size_one_mixed_step_against_oracle(L, O, kind, n, deg):
    """The benchmark sizes (100,352 triangles, P2 and P3; 1024^2 and 2048^2 squares), in
    the launch configuration the autotuner picks for them, from a random
    near-vacuum state with every limiter active: one mixed step against the
    oracle's step, element by element within the FP32 budget, and positive."""
    bc = 2
    s = solver(L, kind, deg, n, bc=(bc,) * 4, tri_bc=bc if kind == TRI else None)
    so = oracle_solver(O, kind, deg, n, bc=(bc,) * 4, tri_bc=bc if kind == TRI else None)
    Q0 = synth.random_modal_state(s.N, s.ML, seed=77 + n, amp=0.3, rho_range=(0.01, 3.0), p_range=(0.001, 3.0))
    Q0[:, :, 1:] = Q0[:, :, 1:].astype(np.float32)
    scratch = L.new_state(s, torch.from_numpy(Q0).cuda())
    L.lxw_autotune(s, scratch, 0.3, reps=1)
    Qo = Q0.copy(); do = so.step(Qo, cfl=0.3)
    st = L.new_state(s, torch.from_numpy(Q0).cuda())
    d = L.lxw_step(s, st, 0.0, 0.3, diag=True)
    Qg = L.to_q64(s, st).cpu().numpy()
    assert d["status"] == 0 and do["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0
    assert d["n_mom"] > 0 and d["n_sc"] > 0                          # the limiters did act
    # s is the largest FP32 speed over ~10^7 point values; the pressure inside
    # c = sqrt(gamma p / rho) cancels (E - |m|^2 / 2 rho), so the FP32 error at
    # the argmax point grows like 1e-7 E / p.  (Positivity needs s only above
    # the averages' speeds: FP32 to 1e-7 under the 1e-5 inflation.)
    assert abs(d["s"] / do["s"] - 1) < 2e-4
    sc = np.abs(Qo).max(axis=0, keepdims=True) + 1e-3
    assert np.abs(Qg[:, :, 0] - Qo[:, :, 0]).max() < 1e-5 * np.abs(Qo[:, :, 0]).max()
    assert (np.abs(Qg - Qo) / sc).max() < 1e-3
    assert np.abs(Qg - Qo).sum() / np.abs(Qo).sum() < 1e-5


@pytest.mark.parametrize("kind", [QUAD, TRI])
def test_fourth_order_ck_mixed_step_close_to_oracle(L, O, kind):
    """ck_order 4 in the mixed form (FP32 bulk): one step of P3 random data
    within the FP32 budget of the oracle's fourth-order step."""
    bc = 2
    s = solver(L, kind, 3, 10, bc=(bc,) * 4, tri_bc=bc if kind == TRI else None, ck_order=4)
    so = oracle_solver(O, kind, 3, 10, bc=(bc,) * 4, tri_bc=bc if kind == TRI else None, ck_order=4)
    Q0 = synth.random_modal_state(s.N, s.ML, seed=41, amp=0.3)
    Q0[:, :, 1:] = Q0[:, :, 1:].astype(np.float32)
    Qo = Q0.copy(); do = so.step(Qo, cfl=0.3)
    st = L.new_state(s, torch.from_numpy(Q0).cuda())
    d = L.lxw_step(s, st, 0.0, 0.3, diag=True)
    Qg = L.to_q64(s, st).cpu().numpy()
    assert d["status"] == 0 and do["status"] == 0
    sc = np.abs(Qo).max(axis=0, keepdims=True) + 1e-3
    assert np.abs(Qg[:, :, 0] - Qo[:, :, 0]).max() < 1e-5 * np.abs(Qo[:, :, 0]).max()
    assert (np.abs(Qg - Qo) / sc).max() < 1e-3
    assert np.abs(Qg - Qo).sum() / np.abs(Qo).sum() < 1e-5
