"""The learned troubled-cell indicator: GPU network against the FP64 oracle
network (forward and gradient), GPU features and limiter labels against the
oracle's on the same state, training on pairs the method generates, and the
gated step (positivity kept, close to the ungated result).

Tolerances: the GPU network and its gradient are FP32 (relative ~1e-6 per
operation over a 24-64-64-1 network -> 1e-4 of the largest gradient entry);
features are FP32 evaluations of the FP32-rounded state (1e-5 relative)."""
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


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.lib()
    return oracle


def test_forward_and_gradient_match_oracle(L, O):
    net = L.lxw_mlp_create(512, seed=11, stream=torch.cuda.current_stream())
    P = L.lxw_mlp_get_params(net).double().cpu().numpy()
    rng = np.random.default_rng(1)
    X = rng.normal(size=(300, 24)); y = rng.uniform(0, 1, 300)
    loss, g = L.lxw_mlp_loss_grad(net, torch.from_numpy(X).float().cuda(), torch.from_numpy(y).float().cuda())
    yh = L.lxw_mlp_forward(net, torch.from_numpy(X).float().cuda()).double().cpu().numpy()
    lo, go, yo = O.mlp_loss_grad(P, X.astype(np.float32).astype(np.float64), y.astype(np.float32).astype(np.float64))
    assert np.abs(yh - yo).max() < 1e-5
    assert abs(loss - lo) < 1e-5 * max(lo, 1e-3)
    g = g.double().cpu().numpy()
    assert np.abs(g - go).max() < 1e-4 * np.abs(go).max()


def mixed_solver(L, kind, n, shock=True, box=(0.0, 1.0, 0.0, 1.0), bc=(2, 2, 2, 2), deg=2):
    if kind == "tri":
        xy, tv = synth.structured_triangles(n, jitter=0.2, seed=20160129, box=box)
        mesh = L.lxw_mesh_triangles(xy, tv)
    else:
        mesh = L.lxw_mesh_cartesian(n, n, box, bc)
    o = L.lxw_options_default(precision=L.PREC_MIXED, shock_limiter=int(shock), alpha0=50.0)
    return L.lxw_solver_create(mesh, deg, o, stream=torch.cuda.current_stream())


def start(L, s, ic):
    xy = L.lxw_projection_points(s)
    r, u, v, p = ic(xy[..., 0], xy[..., 1])
    prim = torch.from_numpy(np.stack(np.broadcast_arrays(r, u, v, p), axis=-1).copy()).cuda()
    Q = torch.zeros(s.q64_shape, dtype=torch.float64, device="cuda")
    L.lxw_project(s, prim, Q)
    return L.new_state(s, Q)


def test_features_and_labels_match_oracle(L, O):
    s = mixed_solver(L, "tri", 16)
    st = start(L, s, synth.ic_rarefy)
    for _ in range(15):
        L.lxw_step(s, st, 0.0, 0.1)
    A = st.clone(); B = st.clone()
    F, th = L.lxw_step_dump(s, A, 0.1)
    s0 = mixed_solver(L, "tri", 16, shock=False)       # same step up to the shock limiter's input
    L.lxw_step(s0, B, 0.0, 0.1)
    Qpre = L.to_q64(s0, B).cpu().numpy()
    # the limiter saw FP32 averages: round the oracle's input the same way
    Qpre[:, :, 0] = Qpre[:, :, 0].astype(np.float32)
    xy, tv = synth.structured_triangles(16, jitter=0.2, seed=20160129)
    so = O.Solver(O.Mesh.triangles(xy, tv), 2, alpha0=50.0)
    Fo = so.features(Qpre)
    Fg = F.double().cpu().numpy()
    assert np.abs(Fg - Fo).max() < 1e-5 * (1 + np.abs(Fo).max())
    tho = so.shock_limit(Qpre.copy())
    thg = th.cpu().numpy()
    assert (tho < 1).sum() > 5
    assert np.abs(thg - tho).max() < 1e-3
    assert np.mean(np.abs(thg - tho) < 1e-5) > 0.99


def generate(L):
    """(features, theta_sc) pairs from plain mixed runs of the smooth wave,
    the double rarefaction and the blast."""
    Xs, ys = [], []
    runs = [("quad", 32, synth.ic_smooth, (0.0, 1.0, 0.0, 1.0), (0, 0, 0, 0), 30),
            ("tri", 32, synth.ic_rarefy, (0.0, 1.0, 0.0, 1.0), (2, 2, 2, 2), 60),
            ("quad", 48, synth.ic_blast(48), (-1.1, 1.1, -1.1, 1.1), (1, 1, 1, 1), 80)]
    for kind, n, ic, box, bc, steps in runs:
        s = mixed_solver(L, kind, n, box=box, bc=bc)
        st = start(L, s, ic)
        for k in range(steps):
            if k % 4 == 3:
                F, th = L.lxw_step_dump(s, st, 0.1)
                Xs.append(F); ys.append(th.float())
            else:
                L.lxw_step(s, st, 0.0, 0.1)
    return torch.cat(Xs), torch.cat(ys)


def test_training_and_gated_step(L):
    X, y = generate(L)
    n = X.shape[0]
    perm = torch.randperm(n, generator=torch.Generator().manual_seed(0)).cuda()
    X, y = X[perm].contiguous(), y[perm].contiguous()
    ntr = int(0.8 * n)
    net = L.lxw_mlp_create(1024, seed=3, stream=torch.cuda.current_stream())
    l0, _ = L.lxw_mlp_loss_grad(net, X[ntr:ntr + 1024].contiguous(), y[ntr:ntr + 1024].contiguous())
    L.lxw_mlp_train(net, X[:ntr].contiguous(), y[:ntr].contiguous(), epochs=8, batch=512, lr=2e-3)
    Xv, yv = X[ntr:].contiguous(), y[ntr:].contiguous()
    yh = torch.cat([L.lxw_mlp_forward(net, Xv[k:k + 1024].contiguous()) for k in range(0, Xv.shape[0], 1024)])
    mse = torch.mean((yh - yv) ** 2).item()
    print(f"pairs {n}, limited {(y < 1).float().mean().item():.3f}, initial mse {l0:.4f}, held-out mse {mse:.5f}")
    assert mse < 0.5 * l0
    tau = 0.02
    skip = yh >= 1 - tau
    # a skipped cell keeps theta = 1: on held-out data those cells rarely needed strong limiting
    assert skip.float().mean().item() > 0.3
    assert (yv[skip] < 0.5).float().mean().item() < 0.02
    # gated blast run: positivity kept, skipped cells counted, close to the plain run
    res = {}
    for gated in (False, True):
        s = mixed_solver(L, "quad", 48, box=(-1.1, 1.1, -1.1, 1.1), bc=(1, 1, 1, 1))
        if gated:
            L.lxw_solver_set_mlp(s, net, tau)
        st = start(L, s, synth.ic_blast(48))
        skipped = 0
        for _ in range(60):
            d = L.lxw_step(s, st, 0.0, 0.1, diag=True)
            assert d["status"] == 0 and d["min_rho"] > 0 and d["min_p"] > 0
            skipped += d["n_mlp_skip"]
        res[gated] = (L.to_q64(s, st).cpu().numpy(), skipped)
    assert res[True][1] > 0 and res[False][1] == 0
    a, b = res[True][0][:, 0, 0], res[False][0][:, 0, 0]
    rel = np.abs(a - b).sum() / np.abs(b).sum()
    print(f"gated blast: skipped {res[True][1]:.0f} cell-steps, density L1 distance {rel:.2e}")
    assert rel < 2e-2

    # the envelope: training recorded the range of its features exactly
    lo, hi = L.lxw_mlp_get_envelope(net)
    Xt = X[:ntr].cpu().numpy()
    assert np.array_equal(lo, Xt.min(axis=0)) and np.array_equal(hi, Xt.max(axis=0))
    # an empty envelope: the gate trusts no cell, skips none, and the gated
    # step is the plain step bit for bit; unbounded again: it skips
    res = {}
    for mode in ("plain", "empty", "unbounded"):
        s = mixed_solver(L, "quad", 48, box=(-1.1, 1.1, -1.1, 1.1), bc=(1, 1, 1, 1))
        if mode == "empty":
            L.lxw_mlp_set_envelope(net, np.full(24, 100.0), np.full(24, 100.0))
        elif mode == "unbounded":
            L.lxw_mlp_set_envelope(net)
        if mode != "plain":
            L.lxw_solver_set_mlp(s, net, 0.5)
        st = start(L, s, synth.ic_blast(48))
        skipped = 0
        for _ in range(20):
            d = L.lxw_step(s, st, 0.0, 0.1, diag=True)
            assert d["status"] == 0
            skipped += d["n_mlp_skip"]
        res[mode] = (st.clone(), skipped)
    assert res["empty"][1] == 0 and torch.equal(res["empty"][0], res["plain"][0])
    assert res["unbounded"][1] > 0
    L.lxw_mlp_set_envelope(net, lo, hi)
    assert np.array_equal(L.lxw_mlp_get_envelope(net)[0], lo)


def bf16(x):
    """Round float32 values to BF16 (nearest even), returned as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32)


def gate_reference(P, F):
    """The gate's network in float64 on BF16-rounded features, weights and
    hidden layer 1 (the rounding the tensor-core path applies), biases and
    the output layer from BF16 weights: the same operation up to FP32
    accumulation order."""
    W = bf16(P).astype(np.float64)
    W1 = W[:24 * 64].reshape(24, 64); b1 = W[1536:1600]
    W2 = W[1600:1600 + 4096].reshape(64, 64); b2 = W[5696:5760]
    w3 = W[5760:5824]; b3 = W[5824]
    X = bf16(F).astype(np.float64)
    H1 = bf16(np.maximum(X @ W1 + b1, 0.0).astype(np.float32)).astype(np.float64)
    H2 = np.maximum(H1 @ W2 + b2, 0.0)
    return 1.0 / (1.0 + np.exp(-(H2 @ w3 + b3)))


@pytest.mark.parametrize("kind,n,deg", [("tri", 21, 2), ("quad", 19, 2), ("tri", 13, 3), ("quad", 11, 3)])
def test_tensor_core_gate_matches_reference_network(L, kind, n, deg):
    """theta_hat of every cell from the tcgen05 path against the same
    network evaluated in float64 on the features the kernel saw; ragged
    tiles (N not a multiple of 32) included."""
    net = L.lxw_mlp_create(256, seed=17, stream=torch.cuda.current_stream())
    P = L.lxw_mlp_get_params(net).cpu().numpy()
    assert P.size == 5825
    box, bc, ic = ((-1.1, 1.1, -1.1, 1.1), (1, 1, 1, 1), synth.ic_blast(n)) if kind == "quad" else \
        ((0.0, 1.0, 0.0, 1.0), (2, 2, 2, 2), synth.ic_rarefy)
    s = mixed_solver(L, kind, n, box=box, bc=bc, deg=deg)
    L.lxw_solver_set_mlp(s, net, 0.0)                     # tau 0: only theta_hat >= 1 would skip
    st = start(L, s, ic)
    for _ in range(3):
        L.lxw_step(s, st, 0.0, 0.1)
    g, F = L.lxw_step_gate(s, st, 0.1, features=True)
    g = g.cpu().numpy(); F = F.cpu().numpy()
    asked = ~np.isnan(g)
    assert asked.sum() == s.N
    ref = gate_reference(P, F)
    # FP32 accumulation of 24 + 64 BF16 products: ~1e-6 relative in z, sigmoid' <= 1/4.
    # The first hidden layer is rounded to BF16 after an FP32 (tensor core) or
    # float64 (here) sum: where the two sums straddle a BF16 rounding boundary one
    # hidden unit differs by one BF16 ulp (2^-8 relative), which moves theta_hat by
    # at most ulp * |h| * sum_n |W2 w3| / 4, a few 1e-3 for these weights.
    d = np.abs(g - ref)
    assert np.mean(d < 2e-5) > 0.99, np.sort(d)[-5:]
    assert d.max() < 5e-3, d.max()
    assert g.std() > 1e-3                                 # the cells do not all give one value


def test_gate_wait_expiry_takes_the_timeout_path(L):
    """The gate's bounded device wait made to run out (a short wait on a
    barrier nothing arrives at, set from the host): the step returns
    LXW_ERR_TIMEOUT, its state equals the ungated step's bit for bit (every
    CTA falls back to the plain limiter), and the next step, with the normal
    bound, is clean and gated again."""
    net = L.lxw_mlp_create(256, seed=9, stream=torch.cuda.current_stream())   # unbounded envelope
    res = {}
    for mode in ("plain", "gated_timeout"):
        s = mixed_solver(L, "quad", 48, box=(-1.1, 1.1, -1.1, 1.1), bc=(1, 1, 1, 1))
        st = start(L, s, synth.ic_blast(48))
        for _ in range(10):
            L.lxw_step(s, st, 0.0, 0.1)                  # a front for the network to rule on
        if mode == "gated_timeout":
            L.lxw_solver_set_mlp(s, net, 0.999)         # skips nearly every cell it rules on
            L.lxw_solver_set_gate_wait_test(s, 1000)
        d = L.lxw_step(s, st, 0.0, 0.1, diag=True)
        res[mode] = (st.clone(), d)
        if mode == "gated_timeout":
            assert d["return_status"] == L.ERR_TIMEOUT and d["status"] & 8 and d["n_mlp_skip"] == 0
            L.lxw_solver_set_gate_wait_test(s, 0)
            d2 = L.lxw_step(s, st, 0.0, 0.1, diag=True)
            assert d2["return_status"] == L.OK and d2["status"] == 0 and d2["n_mlp_skip"] > 0
    assert res["plain"][1]["return_status"] == L.OK
    assert torch.equal(res["gated_timeout"][0], res["plain"][0])


@pytest.mark.parametrize("b3", [-30.0, 30.0])
def test_gated_step_at_one_million_triangles_against_oracle(L, O, b3):
    """The learned-indicator configuration's triangle mesh (708x708x2 =
    1,002,528 jittered P2 triangles, the bench's mesh and options), one gated
    mixed step from near-vacuum data with every limiter active, element by
    element against the oracle.  The network's output bias is pinned so that
    its verdict is known: b3 = -30 gives theta_hat ~ 0 (next to nothing
    skipped: the state is the oracle's step within the FP32 budget); b3 = +30
    gives theta_hat ~ 1 (next to every cell the exact screen leaves is
    skipped).  Cells with theta_hat >= 1 - tau carry the oracle's step
    without the shock limiter, the others its step with it; the averages,
    which the shock limiter never moves, are the oracle's everywhere."""
    n = 708
    xy, tv = synth.structured_triangles(n, jitter=0.2, seed=20160129)
    s = L.lxw_solver_create(L.lxw_mesh_triangles(xy, tv), 2, L.lxw_options_default(precision=L.PREC_MIXED),
                            stream=torch.cuda.current_stream())
    assert s.N == 1_002_528
    net = L.lxw_mlp_create(256, seed=29, stream=torch.cuda.current_stream())
    P = L.lxw_mlp_get_params(net)
    P[5824] = b3
    L.lxw_mlp_set_params(net, P)
    L.lxw_solver_set_mlp(s, net, 0.01)
    # near-vacuum random data in the first eighth of the cells (a band of the
    # mesh), a uniform state (rho 1, p 0.4, at rest) in the others: the exact
    # screen clears the uniform cells away from the band and none in it
    Q0 = synth.random_modal_state(s.N, s.ML, seed=5708, amp=0.3, rho_range=(0.01, 3.0), p_range=(0.001, 3.0))
    calm = np.arange(s.N) >= s.N // 8
    Q0[calm] = 0.0
    Q0[calm, 0, 0] = 1.0
    Q0[calm, 3, 0] = 0.4 / 0.4
    Q0[:, :, 1:] = Q0[:, :, 1:].astype(np.float32)
    st = L.new_state(s, torch.from_numpy(Q0).cuda())
    st2 = st.clone()
    g = L.lxw_step_gate(s, st, 0.3).cpu().numpy()
    Qg = L.to_q64(s, st).cpu().numpy()
    # the ordinary gated step (the plain kernel screens and lists, the gate
    # kernel takes the listed cells) gives the state of the full scan above
    d2 = L.lxw_step(s, st2, 0.0, 0.3, diag=True)
    assert torch.equal(st, st2)
    asked = ~np.isnan(g)
    skipped = asked & (g >= 0.99)
    assert asked.sum() >= 0.99 * s.N               # theta_hat is reported for every cell
    om = O.Mesh.triangles(xy, tv)
    Qa = Q0.copy(); da = O.Solver(om, 2).step(Qa, cfl=0.3)
    assert da["n_sc"] > 0 and da["status"] == 0
    sc = np.abs(Qa).max(axis=0, keepdims=True) + 1e-3
    # averages: the oracle's everywhere (the shock limiter never moves them)
    assert np.abs(Qg[:, :, 0] - Qa[:, :, 0]).max() < 1e-5 * np.abs(Qa[:, :, 0]).max()
    Qb = Q0.copy(); O.Solver(om, 2, shock_limiter=False).step(Qb, cfl=0.3)
    # cells the gate did not skip: the oracle's step; skipped ones: without the
    # shock limiter (a cell the exact screen clears has theta = 1 in the
    # oracle, so there both agree whatever theta_hat says)
    if (~skipped).any():
        assert (np.abs(Qg[~skipped] - Qa[~skipped]) / sc).max() < 1e-3
    if skipped.any():
        assert (np.abs(Qg[skipped] - Qb[skipped]) / sc).max() < 1e-3
    if b3 < 0:
        assert skipped.sum() <= 0.01 * asked.sum() and d2["n_mlp_skip"] <= 0.01 * s.N
        assert np.abs(Qg - Qa).sum() / np.abs(Qa).sum() < 1e-5
    else:
        assert skipped.sum() >= 0.99 * asked.sum() and d2["n_mlp_skip"] > 0
        # the skipped cells include cells the oracle's shock limiter does change
        moved = np.abs(Qa[skipped, :, 1:] - Qb[skipped, :, 1:]).max(axis=(1, 2)) > 1e-3 * sc[0, :, 1:].max()
        assert moved.sum() > 0


@pytest.mark.parametrize("kind,n,deg", [("quad", 48, 2), ("tri", 21, 3)])
def test_gate_scan_and_list_forms_agree(L, kind, n, deg):
    """The gated limiter's two forms -- the gate kernel screening every cell
    (gate_scan 1) or the plain kernel screening and listing the uncleared
    cells for it (gate_scan 0, two launches) -- give the same states and skip
    counts bit for bit over several steps, with a network that skips most of
    the cells it rules on; the autotuner reports the form it keeps."""
    net = L.lxw_mlp_create(256, seed=9, stream=torch.cuda.current_stream())
    box, bc, ic = ((-1.1, 1.1, -1.1, 1.1), (1, 1, 1, 1), synth.ic_blast(n)) if kind == "quad" else \
        ((0.0, 1.0, 0.0, 1.0), (2, 2, 2, 2), synth.ic_rarefy)
    states, skips = [], []
    for scan in (0, 1):
        if kind == "tri":
            xy, tv = synth.structured_triangles(n, jitter=0.2, seed=20160129, box=box)
            mesh = L.lxw_mesh_triangles(xy, tv)
        else:
            mesh = L.lxw_mesh_cartesian(n, n, box, bc)
        o = L.lxw_options_default(precision=L.PREC_MIXED, alpha0=50.0, gate_scan=scan)
        s = L.lxw_solver_create(mesh, deg, o, stream=torch.cuda.current_stream())
        L.lxw_solver_set_mlp(s, net, 0.999)
        assert L.lxw_step_launches(s) == (5 if scan else 6)
        assert L.lxw_solver_get_options(s)["gate_scan"] == scan
        st = start(L, s, ic)
        sk = 0
        for _ in range(12):
            d = L.lxw_step(s, st, 0.0, 0.1, diag=True)
            assert d["return_status"] == L.OK
            sk += d["n_mlp_skip"]
        states.append(st)
        skips.append(sk)
    assert skips[0] == skips[1] and skips[0] > 0
    assert torch.equal(states[0], states[1])
    res = L.lxw_autotune(s, st.clone(), 0.1, reps=1)
    assert res["gate_scan"] in (0, 1)
    assert L.lxw_step_launches(s) == (5 if res["gate_scan"] else 6)
