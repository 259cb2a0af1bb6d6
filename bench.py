#!/usr/bin/env python
"""Throughput of the LxW-DG time step on the GPU, in DOF-updates/s.

A step is one pass of the whole hot path (moment limiter, wave speed, CK
time-averaged flux and volume integral, edge fluxes, flux limiter, blended
update, shock limiter) over the workload.  Default workload: the learned-
indicator configuration -- a 2048x2048 Cartesian P2 point-energy blast
(4,194,304 cells) and 708x708 squares split into 1,002,528 jittered P2
triangles with the two-rarefaction near-vacuum data; one step is one step of
each, the mixed form with the MLP-gated shock limiter timed against the
plain FP64 form on the same meshes.  The 224x224x2 = 100,352-triangle
rarefaction (the unstructured configuration of the FP64-vs-mixed
comparison) is measured beside it.  Inputs are synthetic and resident in
HBM before timing; the L2 is flushed (256 MB write) between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica of the workload
(the problems are independent; no collective on the data path) and the
slowest rank's time counts.  --impl reference times the FP64 CPU oracle,
the slow plain reference of this repository, on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "DOF-updates/s, LxW-DG Euler P2: mixed+learned vs plain FP64 GPU at equal L1 error"
UNIT = "DOF-updates/s"

WORKLOADS = {
    "rarefy": dict(kind="tri", n=224, deg=2, cfl=0.1, ic=synth.ic_rarefy,
                   desc="rarefaction: 224x224x2 = 100,352 jittered triangles, P2, rho=1 p=0.4 u=-+2, transparent"),
    "blast": dict(kind="quad", n=1024, deg=2, cfl=0.1, ic=None, bc=(1, 1, 1, 1), box=(-1.1, 1.1, -1.1, 1.1),
                  desc="blast: 1024x1024 Cartesian, P2, point energy 0.979264 in the 4 centre cells, reflective"),
    "smooth": dict(kind="quad", n=32, deg=2, cfl=0.1, ic=synth.ic_smooth,
                   desc="smooth: 32x32 periodic Cartesian, P2, advected density wave"),
    "rarefy_p3": dict(kind="tri", n=224, deg=3, cfl=0.1, ic=synth.ic_rarefy,
                      desc="rarefaction: 224x224x2 = 100,352 jittered triangles, P3, rho=1 p=0.4 u=-+2, transparent"),
    "rarefy1m": dict(kind="tri", n=724, deg=2, cfl=0.1, ic=synth.ic_rarefy,
                     desc="rarefaction: 724x724x2 = 1,048,352 jittered triangles, P2, rho=1 p=0.4 u=-+2, transparent"),
    "rarefy708": dict(kind="tri", n=708, deg=2, cfl=0.1, ic=synth.ic_rarefy,
                      desc="rarefaction: 708x708x2 = 1,002,528 jittered triangles, P2, rho=1 p=0.4 u=-+2, transparent"),
    "blast2048": dict(kind="quad", n=2048, deg=2, cfl=0.1, ic=None, bc=(1, 1, 1, 1), box=(-1.1, 1.1, -1.1, 1.1),
                      desc="blast: 2048x2048 Cartesian, P2, point energy 0.979264 in the 4 centre cells, reflective"),
    "sedov": dict(kind="disk", n=136270, deg=2, cfl=0.1, ic=synth.ic_sedov_disk(136270),
                  desc="Sedov blast on a disk: 136,270 Delaunay triangles of the circle of radius 1.1 "
                       "(jittered triangular lattice), P2, point energy 0.979264 inside r_d, reflective rim"),
    "diffraction": dict(kind="step", nx=390, ny=330, deg=2, cfl=0.1, ic=synth.ic_diffraction,
                        box=synth.DIFFRACTION_BOX, bc=synth.DIFFRACTION_BC,
                        desc="shock diffraction: Mach 5.09 over a step, 390x330 Cartesian on [0,13]x[0,11] less the "
                             "step [0,1]x[0,6] (123,300 cells), P2, inflow above the step, walls on it, "
                             "transparent elsewhere"),
}
# Workloads made of several meshes: one step is one step of each part.
CONFIGS = {
    "config5": dict(parts=("blast2048", "rarefy708"),
                    desc="learned-indicator configuration: 2048x2048 Cartesian P2 blast (4,194,304 cells, point energy "
                         "0.979264 in the 4 centre cells, reflective) and 708x708x2 = 1,002,528 jittered P2 "
                         "triangles (rho=1 p=0.4 u=-+2, transparent); one step = one step of each"),
}


def parts_of(name):
    return CONFIGS[name]["parts"] if name in CONFIGS else (name,)


def desc_of(name):
    return CONFIGS[name]["desc"] if name in CONFIGS else WORKLOADS[name]["desc"]


ENSEMBLE = dict(count=256, lo=32, hi=256, seed=4242, deg=2, cfl=0.3,
                desc="ensemble: 256 independent Cartesian problems n_p x n_p, n_p ~ U{32..256} (seed 4242), "
                     "P2, four-quadrant Riemann data per problem seed, transparent")

# Algorithmic FP64 work per element of the CK kernel (P2): the modal <->
# point contractions (q at 21 points 1008, two projections 1728, q_t and q_tt
# at 21 points 2016 each, volume integral 864) plus the pointwise flux,
# Jacobian and Hessian products and F_T assembly (~250 flop at each of 21
# points).  Triangles (9 interior + 9 edge points) scale the point terms.
def ck_flops_per_element(kind, deg):
    ML = (deg + 1) * (deg + 2) // 2
    NQ = (deg + 1) ** 2
    NE = (3 if kind in ("tri", "disk") else 4) * (deg + 1)
    npt = NQ + NE
    contract = 2 * 4 * ML * npt + 2 * 2 * 2 * 4 * ML * NQ + 2 * (2 * 2 * 4 * ML * npt) + 2 * 2 * 4 * ML * NQ
    return contract + 250 * npt


FP64_PEAK_TFLOPS = 1.25   # GB300 nominal dense FP64 (recipe table; the FMA probe measures 1.253)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 80.5: SMs x FP32 lanes x 2 flop x max SM clock

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the CK kernel, from ncu captures, per (workload, form): the bytes, the first
# 16 hex digits of the SHA-256 of the kernel source the capture ran, and the
# elements of the captured mesh when it was a smaller mesh of the same kind
# scaled to the workload by the element count (the traffic of this kernel is
# proportional to it).  A capture of another kernel source reads as None.
CK_TRAFFIC = {
    ("blast2048", "mixed"): {"bytes": 151_320_576 + 433_108_736, "source": "d3d1fe0e7a0d7dc1", "captured_elements": 1_048_576},
    ("blast", "mixed"): {"bytes": 151_320_576 + 433_108_736, "source": "d3d1fe0e7a0d7dc1"},
    ("rarefy708", "mixed"): {"bytes": 136_541_696 + 312_284_160, "source": "d3d1fe0e7a0d7dc1"},
}


def kernel_source_hash(mixed):
    """Hash of the source the CK kernel is built from: for the mixed form the
    part of lxw_kernels_mx.cu up to the edge kernel (tables, FP32 physics,
    the moment and CK kernels), so that edits of the later kernels keep a
    capture of k_ck_mx current; the whole file for the FP64 form."""
    import hashlib
    src = os.path.join(ROOT, "paper_1601_08145_gb300", "csrc", "lxw_kernels_mx.cu" if mixed else "lxw_kernels.cu")
    text = open(src, "rb").read()
    if mixed:
        text = text[:text.index(b"// ---------------------------------------------------------- k_edge_mx")]
    return hashlib.sha256(text).hexdigest()[:16]


def ck_traffic(name, mixed, elements):
    rec = CK_TRAFFIC.get((name, "mixed" if mixed else "fp64"))
    if rec is None or rec["source"] != kernel_source_hash(mixed):
        return None
    return rec["bytes"] * elements / rec.get("captured_elements", elements)


def build_workload(L, name, stream, mixed):
    return build_solver(L, WORKLOADS[name], stream, mixed)


def build_solver(L, w, stream, mixed):
    if w["kind"] == "tri":
        xy, tv = synth.structured_triangles(w["n"], jitter=0.2, seed=20160129)
        mesh = L.lxw_mesh_triangles(xy, tv)
    elif w["kind"] == "disk":
        xy, tv = synth.disk_triangles(w["n"])
        mesh = L.lxw_mesh_triangles(xy, tv, np.full((w["n"], 3), L.BC_REFLECT, np.int32))
    elif w["kind"] == "step":
        mesh = L.lxw_mesh_cartesian_masked(w["nx"], w["ny"], w["box"], w["bc"],
                                           synth.diffraction_mask(w["nx"], w["ny"]), L.BC_REFLECT)
    else:
        mesh = L.lxw_mesh_cartesian(w["n"], w["n"], w.get("box", (0.0, 1.0, 0.0, 1.0)), w.get("bc", (0, 0, 0, 0)))
    opt = L.lxw_options_default(precision=L.PREC_MIXED if mixed else L.PREC_FP64)
    sol = L.lxw_solver_create(mesh, w["deg"], opt, stream=stream)
    if w["kind"] == "step":
        L.lxw_solver_set_inflow(sol, synth.normal_shock_state(synth.DIFFRACTION_MACH))
    return w, sol


def oracle_solver(w):
    """The oracle's solver and initial state for a workload."""
    from oracle import oracle as O
    if w["kind"] == "tri":
        xy, tv = synth.structured_triangles(w["n"], jitter=0.2, seed=20160129)
        m = O.Mesh.triangles(xy, tv)
    elif w["kind"] == "disk":
        xy, tv = synth.disk_triangles(w["n"])
        m = O.Mesh.triangles(xy, tv, np.full((w["n"], 3), O.REFLECT, np.int32))
    elif w["kind"] == "step":
        m = O.Mesh.cartesian_masked(w["nx"], w["ny"], w["box"], w["bc"], synth.diffraction_mask(w["nx"], w["ny"]),
                                    O.REFLECT)
    else:
        m = O.Mesh.cartesian(w["n"], w["n"], w.get("box", (0.0, 1.0, 0.0, 1.0)), w.get("bc", (0, 0, 0, 0)))
    s = O.Solver(m, w["deg"])
    if w["kind"] == "step":
        s.set_inflow(synth.normal_shock_state(synth.DIFFRACTION_MACH))
    return s, s.project_fn(w["ic"] or synth.ic_blast(w["n"]))


def half_resolution(w):
    if w["kind"] == "step":
        return dict(w, nx=w["nx"] // 2, ny=w["ny"] // 2)
    if w["kind"] == "disk":   # half the spacing: a quarter of the cells, r_d of that mesh
        return dict(w, n=w["n"] // 4, ic=synth.ic_sedov_disk(w["n"] // 4))
    return dict(w, n=w["n"] // 2)


def project(L, sol, w):
    import torch
    ic = w["ic"] or synth.ic_blast(w["n"])
    xy = L.lxw_projection_points(sol)
    r, u, v, p = ic(xy[..., 0], xy[..., 1])
    prim = torch.from_numpy(np.stack(np.broadcast_arrays(r, u, v, p), axis=-1).copy()).cuda()
    Q = torch.empty(sol.q64_shape, dtype=torch.float64, device="cuda")
    L.lxw_project(sol, prim, Q)
    return L.new_state(sol, Q) if sol.mixed else Q


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.lines, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=lambda: [self.lines.append(l) for l in self.proc.stdout], daemon=True).start()
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            self.proc.wait(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


TRAINING_RUNS = (("smooth", 40, 4), ("rarefy", 60, 6), ("blast", 40, 10), ("diffraction", 60, 6), ("sedov", 60, 6))


def train_indicator(L, stream, tau=0.01):
    """Train the troubled-cell MLP on the GPU from (features, limiter theta)
    pairs that plain mixed runs of the benchmark configurations produce (the
    smooth wave 32x32, the rarefaction on 100,352 triangles, the blast on
    1024x1024, the shock diffraction on 123,300 squares, the Sedov disk on
    136,270 triangles); every limited pair is kept, the others are subsampled
    to about 400k, and the limited pairs are repeated to a quarter of the set.
    Returns the net and a summary (held-out numbers on 20 % of the pairs)."""
    import torch
    gen = torch.Generator(device="cuda").manual_seed(7)
    Xs, ys = [], []
    for name, steps, every in TRAINING_RUNS:
        w, sol = build_workload(L, name, stream, True)
        st = project(L, sol, w)
        for k in range(steps):
            if k % every == every - 1:
                F, th = L.lxw_step_dump(sol, st, w["cfl"])
                Xs.append(F); ys.append(th.float())
            else:
                L.lxw_step(sol, st, 0.0, w["cfl"])
    X = torch.cat(Xs); y = torch.cat(ys)
    lim = y < 1.0
    n_un = int((~lim).sum().item())
    keep = lim | (torch.rand(X.shape[0], device="cuda", generator=gen) < min(1.0, 4e5 / max(n_un, 1)))
    X, y = X[keep], y[keep]
    perm = torch.randperm(X.shape[0], device="cuda", generator=gen)
    X, y = X[perm].contiguous(), y[perm].contiguous()
    nval = X.shape[0] // 5
    Xv, yv, Xt, yt = X[:nval], y[:nval], X[nval:], y[nval:]
    lim = yt < 1.0
    reps = max(1, int(0.25 * Xt.shape[0] / max(int(lim.sum().item()), 1)))
    Xt = torch.cat([Xt] + [Xt[lim]] * (reps - 1)); yt = torch.cat([yt] + [yt[lim]] * (reps - 1))
    perm = torch.randperm(Xt.shape[0], device="cuda", generator=gen)
    Xt, yt = Xt[perm].contiguous(), yt[perm].contiguous()
    net = L.lxw_mlp_create(1024, seed=3, stream=stream)
    loss = L.lxw_mlp_train(net, Xt, yt, epochs=6, batch=512, lr=2e-3)
    yh = torch.cat([L.lxw_mlp_forward(net, Xv[k:k + 1024].contiguous()) for k in range(0, Xv.shape[0], 1024)])
    strong = yv < 1.0 - 2 * tau
    missed = ((yh >= 1.0 - tau) & strong).sum().item() / max(int(strong.sum().item()), 1)
    return net, {"pairs_generated": int(keep.numel()), "pairs_kept": int(X.shape[0]),
                 "limited_fraction_kept": float((y < 1).float().mean().item()),
                 "limited_repeat": reps, "final_batch_mse": loss,
                 "heldout_mse": float(torch.mean((yh - yv) ** 2).item()),
                 "heldout_skip_fraction": float((yh >= 1.0 - tau).float().mean().item()),
                 "heldout_missed_strongly_limited": missed}


def cpu_baseline(name, budget_s=10.0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same
    workload: whole steps of each part, at least one and up to 5 per part
    (the step window of the measurement plan) or the time budget."""
    from oracle import oracle as O
    dofs, secs, ks = 0.0, 0.0, []
    for part in parts_of(name):
        w = WORKLOADS[part]
        s, Q = oracle_solver(w)
        s.step(Q, cfl=w["cfl"])          # untimed first step (page-in)
        t0 = time.perf_counter(); k = 0
        while k < 1 or (time.perf_counter() - t0 < budget_s / len(parts_of(name)) and k < 5):
            s.step(Q, cfl=w["cfl"]); k += 1
        secs += time.perf_counter() - t0
        dofs += s.N * 4 * s.ML * k
        ks.append(f"{k} full steps of {part} ({s.N} elements)")
        del s, Q
    out = {"value": dofs / secs, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
           "sample": "; ".join(ks) + f" from the initial data, {secs:.1f} s"}
    # the same oracle on one core: the reference arm in a child process with one OpenMP thread
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1", RANK="0", WORLD_SIZE="1")
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", name,
                            "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=900)
        one = json.loads(r.stdout.strip().splitlines()[-1])
        out["one_core"] = {"value": one["value"], "cores": one["cpu_baseline"]["cores"],
                           "sample": "1 full step of each part, OMP_NUM_THREADS=1"}
    except Exception as e:   # the multi-core number stands on its own
        out["one_core"] = {"value": None, "error": str(e)[:200]}
    return out, ks, secs


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores,
    on the same workload (every part), K timed steps after W warm-up steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    if args.workload == "blast3d":
        # the 3D oracle on a 48^3 sample of the blast (its work arrays, ~15 KB
        # per cell, would take 13 GB of host memory at 96^3)
        b = BLAST3D
        box = (-b["half_width"], b["half_width"]) * 3
        so = O.Solver3(O.Mesh3(48, 48, 48, box, (1,) * 6), b["deg"])
        Q = so.project_fn(synth.ic_blast3d(48, b["half_width"]))
        sols = [(b, so, Q)]
        nv = 5
    elif args.workload == "blast3t":
        # the same blast on a 24^3-box sample of the tetrahedral mesh
        b = BLAST3T
        box = (-b["half_width"], b["half_width"]) * 3
        xo, to, vo = synth.tet_mesh(24, box=box)
        so = O.Solver3(O.Mesh3.tets(xo, to, vo, np.full((len(to), 4), 1, dtype=np.int32)), b["deg"])
        Q = so.project_fn(synth.ic_blast3d(24, b["half_width"]))
        sols = [(b, so, Q)]
        nv = 5
    else:
        sols = [(WORKLOADS[p],) + oracle_solver(WORKLOADS[p]) for p in parts_of(args.workload)]
        nv = 4
    for _ in range(args.warmup):
        for w, s, Q in sols:
            s.step(Q, cfl=w["cfl"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for w, s, Q in sols:
            s.step(Q, cfl=w["cfl"])
    dt = time.perf_counter() - t0
    dof = sum(s.N * nv * s.ML for _, s, _ in sols)
    val = dof * args.steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": {"blast3d": BLAST3D["desc"], "blast3t": BLAST3T["desc"]}.get(args.workload)
                      or desc_of(args.workload),
                      "elements": sum(s.N for _, s, _ in sols), "degree": 2,
                      "form": "FP64 CPU oracle"},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                            "sample": f"{args.steps} full steps of every part after {args.warmup} warm-up steps"},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_ensemble(args):
    """Batched independent problems: one solver over the union (one launch per
    phase, one graph per step, autotuned work list) against one solver per
    problem stepped in turn."""
    import torch
    from paper_1601_08145_gb300 import build, lxw as L
    build.build()
    e = ENSEMBLE
    sizes = synth.ensemble_sizes(e["count"], e["lo"], e["hi"], e["seed"])
    stream = torch.cuda.current_stream()
    meshes, ics = [], []
    for k, n in enumerate(sizes):
        meshes.append(L.lxw_mesh_cartesian(int(n), int(n), (0.0, 1.0, 0.0, 1.0), (2, 2, 2, 2)))
        ics.append(synth.ic_quadrants(e["seed"] + 1 + k))
    def proj(sol, ic):
        xy = L.lxw_projection_points(sol)
        r, u, v, p = ic(xy[..., 0], xy[..., 1])
        prim = torch.from_numpy(np.stack(np.broadcast_arrays(r, u, v, p), axis=-1).copy()).cuda()
        Q = torch.empty(sol.q64_shape, dtype=torch.float64, device="cuda")
        L.lxw_project(sol, prim, Q)
        return Q
    mopt = L.lxw_options_default(precision=L.PREC_MIXED)
    singles = [L.lxw_solver_create(m, e["deg"], mopt, stream=stream) for m in meshes]
    Q = torch.cat([proj(s, ic) for s, ic in zip(singles, ics)])
    b = L.lxw_batch_create(meshes, e["deg"], mopt, stream=stream)
    st = L.new_state(b, Q)
    tune = L.lxw_autotune(b, st, e["cfl"], reps=3)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    L.lxw_run(b, st, max(args.warmup, 3), e["cfl"])
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start(); time.sleep(0.5)
    torch.cuda.synchronize()
    total_ms = time_steps(L, b, st, e["cfl"], args.steps, flush)
    clk = clocks.stop()
    phases = [L.lxw_profile_step(b, st, e["cfl"]) for _ in range(3)]
    dof = b.N * 4 * b.ML
    # one solver per problem, each its own graph-replayed step, in turn
    sstates = [L.new_state(s, Q[b.offsets[k]:b.offsets[k + 1]].contiguous()) for k, s in enumerate(singles)]
    for s, x in zip(singles, sstates):
        L.lxw_run(s, x, 1, e["cfl"])
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True); ev1 = torch.cuda.Event(enable_timing=True)
    nrep = max(2, args.steps // 4)
    ev0.record()
    for _ in range(nrep):
        for s, x in zip(singles, sstates):
            L.lxw_run(s, x, 1, e["cfl"])
    ev1.record(); torch.cuda.synchronize()
    per_ms = ev0.elapsed_time(ev1) / nrep
    out = {"metric": METRIC, "value": dof * args.steps / (total_ms / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
           "data": "synthetic",
           "config": {"workload": e["desc"], "elements": b.N, "problems": len(sizes), "degree": e["deg"],
                      "form": "mixed, batched", "cfl": e["cfl"], "l2": "flushed between timed steps"},
           "autotune": tune,
           "phases_ms": {k: statistics.mean(p[k] for p in phases) for k in phases[0]},
           "unbatched": {"value": dof / (per_ms / 1e3), "ms_per_step": per_ms,
                         "how": "one solver per problem, each step a graph launch, problems in turn"},
           "batching_speedup": per_ms / (total_ms / args.steps),
           "gpu_launches": args.steps * L.lxw_step_launches(b),
           "clocks": clk}
    print(json.dumps(out))


BLAST3D = dict(n=96, deg=2, cfl=0.1, half_width=1.1,
               desc="3D blast: 96^3 = 884,736 Cartesian P2 cells of [-1.1,1.1]^3, point energy 0.979264 in the "
                    "8 centre cells, reflective walls (FP64 form)")


BLAST3T = dict(n=48, deg=2, cfl=0.1, half_width=1.1,
               desc="3D blast on tetrahedra: 48^3 boxes of [-1.1,1.1]^3 cut into 6 Kuhn tetrahedra = 663,552 P2 "
                    "cells, point energy 0.979264 in the 48 cells around the origin, reflective walls (FP64 form)")


# DRAM bytes (read + write) of one launch of the mixed forms' FP32 CK kernel from an ncu
# capture of the same blast on a smaller mesh (--n3 32 / 64), scaled by the cells (the
# kernel's traffic is per cell: the state read and written back, the FP32 traces), valid
# while the source the kernel is built from is unchanged
CK3_TRAFFIC = {
    "blast3t": {"bytes": 125_647_104 + 302_418_688, "captured_elements": 196_608, "source": "45533b02a27e26d1"},
    "blast3d": {"bytes": 154_067_712 + 615_788_544, "captured_elements": 262_144, "source": "e01c9701d787f53b"},
}


def ck3_source_hash(tet):
    """Hash of the 3D helpers and of the kernel file up to its face kernel."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1601_08145_gb300", "csrc")
    tu, marker = (("lxw_kernels3t.cu", b"// ------------------------------------------------------------ k3t_face") if tet
                  else ("lxw_kernels3d.cu", b"// ------------------------------------------------------------ k3_face"))
    text = open(os.path.join(csrc, tu), "rb").read()
    return hashlib.sha256(open(os.path.join(csrc, "lxw_flux3.cuh"), "rb").read() + text[:text.index(marker)]).hexdigest()[:16]


def ck3t_flops_per_element(deg):
    """Algorithmic flop of k3t_ck per tetrahedron (an FMA counts 2), the
    hexahedral count with NPT = NQ + 4 n^2 points and, at each interior
    point of every pass, the contravariant flux G_a = sum_d Ji[a][d] F_d (45
    FMA) in place of the three axis scalings; a face point evaluates q, q_t,
    q_tt and only the normal component an_k . F_T (the normal flux and its
    derivatives, ~200)."""
    n = deg + 1
    NQ, NF = n ** 3, n * n
    ML = (deg + 1) * (deg + 2) * (deg + 3) // 6
    p1 = NQ * (2 * 5 * ML + 40 + 90 + 2 * 15 * ML)
    p2 = NQ * (2 * 10 * ML + 70 + 90 + 2 * 15 * ML)
    p3 = NQ * (2 * 15 * ML + 320 + 90 + 2 * 15 * (ML - 1)) + 4 * NF * (2 * 15 * ML + 200)
    return p1 + p2 + p3


def ck3_flops_per_element(deg):
    """Algorithmic FP64 flop of k3_ck per cell (an FMA counts 2): with n =
    deg + 1, NQ = n^3 interior and 6 n^2 face points, ML modes, 5 variables.
    Pass 1: q at the interior points (5 ML FMA), the flux (~40), the three
    weighted-table sums (15 ML FMA + 15).  Pass 2: q and q_t (10 ML FMA),
    F'(q) q_t (~70), three table sums (15 ML FMA + 15).  Pass 3 at the
    interior points: q, q_t, q_tt (15 ML FMA), F, F' q_t, F'' (q_t, q_t),
    F' q_tt and F_T (~320), the volume sums (15 (ML-1) FMA + 15); at the face
    points: q, q_t, q_tt and only the normal component of F_T (the normal
    flux and its derivatives, ~200)."""
    n = deg + 1
    NQ, NF = n ** 3, n * n
    ML = (deg + 1) * (deg + 2) * (deg + 3) // 6
    p1 = NQ * (2 * 5 * ML + 40 + 2 * 15 * ML + 15)
    p2 = NQ * (2 * 10 * ML + 70 + 2 * 15 * ML + 15)
    p3 = NQ * (2 * 15 * ML + 320) + 6 * NF * (2 * 15 * ML + 200) + NQ * (2 * 15 * (ML - 1) + 15)
    return p1 + p2 + p3


def run_blast3d(args):
    """The 3D forms on the 3D point-energy blast (Cartesian hexahedra, or with
    --workload blast3t the same blast on Kuhn tetrahedra): the mixed form
    (the line's value) and the FP64 form, each K graph-replayed steps from the
    same projected state bracketed by CUDA events (the state, 265-354 MB,
    exceeds the L2), per-phase times from traced steps, the oracle on a
    sample.  --form mixed / fp64 times one form only."""
    import torch
    from paper_1601_08145_gb300 import build, lxw as L
    build.build()
    tet = args.workload == "blast3t"
    b = BLAST3T if tet else BLAST3D
    if args.n3:   # a smaller mesh of the same blast (profiling captures)
        b = dict(b, n=args.n3, desc=b["desc"] + " -- run here at %d per axis" % args.n3)
    n, hw = b["n"], b["half_width"]
    box = (-hw, hw) * 3
    stream = torch.cuda.current_stream()
    if tet:
        xyz, tets, vid = synth.tet_mesh(n, box=box)
        walls = np.full((len(tets), 4), 1, dtype=np.int32)
        make = lambda o: L.lxw3_solver_create_tets(xyz, tets, vid, b["deg"], face_bc=walls, options=o,  # noqa: E731
                                                   stream=stream)
    else:
        make = lambda o: L.lxw3_solver_create(n, n, n, box, (1,) * 6, b["deg"], o, stream=stream)  # noqa: E731
    forms = {"mixed": L.PREC_MIXED, "fp64": L.PREC_FP64}
    if args.form in forms:
        forms = {args.form: forms[args.form]}
    ic = synth.ic_blast3d(n, hw)
    Q0 = None
    res = {}
    probes = fma_probes()
    flop_cell = (ck3t_flops_per_element if tet else ck3_flops_per_element)(b["deg"])
    for name, prec in forms.items():
        s = make(L.lxw_options_default(precision=prec))
        if Q0 is None:
            xyz3 = L.lxw3_projection_points(s)
            prim = torch.from_numpy(np.stack(np.broadcast_arrays(*ic(xyz3[..., 0], xyz3[..., 1], xyz3[..., 2])),
                                             axis=-1).copy())
            del xyz3
            Q0 = torch.zeros(s.state_shape, dtype=torch.float64, device="cuda")
            L.lxw3_project(s, prim.cuda(), Q0)
            del prim
        Q = Q0.clone()
        L.lxw3_run(s, Q, max(args.warmup, 3), b["cfl"])
        clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
        clocks.start(); time.sleep(0.5)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        d = L.lxw3_run(s, Q, args.steps, b["cfl"], diag=True)
        ev1.record(); torch.cuda.synchronize()
        clk = clocks.stop()
        total_ms = ev0.elapsed_time(ev1)
        phases = [L.lxw3_profile_step(s, Q, b["cfl"]) for _ in range(3)]
        ph = {k: statistics.mean(p[k] for p in phases) for k in phases[0]}
        flops = flop_cell * s.N
        fp32 = name == "mixed"
        peak = FP32_PEAK_TFLOPS if fp32 else 1.25
        roof = {"kernel": ("k3t_ck" if tet else "k3_ck") + ("<float>" if fp32 else "<double>"), "bound": "alu",
                "pipe": "fp32" if fp32 else "fp64", "achieved": flops / (ph["ck"] / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s",
                "peak_source": ("152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz" if fp32
                                else "nominal GB300 FP64 rate (recipe table)"),
                "peak_measured_fma_probe": probes.get("fp32" if fp32 else "fp64"),
                "algorithmic_flops_per_launch": flops, "launch_ms": ph["ck"], "traffic": None}
        rec = CK3_TRAFFIC.get(args.workload)
        if fp32 and rec is not None and rec["source"] == ck3_source_hash(tet):
            roof["traffic"] = rec["bytes"] * s.N / rec["captured_elements"]
            roof["traffic_source"] = "ncu dram__bytes_read+write at %d cells, scaled by the cells" % rec["captured_elements"]
            roof["algorithmic_bytes_per_launch"] = s.N * (5 * s.ML * 8 + 5 * (s.ML - 1) * 8 + (4 if tet else 6) * (
                (b["deg"] + 1) ** 2) * 10 * 4)
        roof["frac"] = roof["achieved"] / peak
        res[name] = {"value": s.N * 5 * s.ML * args.steps / (total_ms / 1e3), "ms_per_step": total_ms / args.steps,
                     "phases_ms": ph, "roofline": roof, "clocks": clk, "launches": args.steps * L.lxw3_step_launches(s) + 1,
                     "positivity_last_step": {"min_rho": d["min_rho"], "min_p": d["min_p"]}, "status_last_step": d["status"],
                     "elements": s.N, "dof": s.N * 5 * s.ML}
        del s
    head = "mixed" if "mixed" in res else "fp64"
    r = res[head]
    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if head == "mixed" else "f64", "data": "synthetic",
           "config": {"workload": b["desc"], "elements": r["elements"], "degree": b["deg"], "cfl": b["cfl"],
                      "form": {"mixed": "mixed (FP32 CK kernel, FP64 state and limiters)", "fp64": "FP64"}[head],
                      "l2": "state (%d MB) larger than the L2" % (r["dof"] * 8 // 10 ** 6),
                      "timing": "graph-replayed steps, CUDA events"},
           "phases_ms": r["phases_ms"], "roofline": r["roofline"],
           "gpu_launches": sum(x["launches"] for x in res.values()),
           "clocks": r["clocks"], "positivity_last_step": r["positivity_last_step"],
           "status_last_step": r["status_last_step"]}
    if len(res) > 1:
        out["fp64_form"] = {k: res["fp64"][k] for k in ("value", "ms_per_step", "phases_ms", "roofline",
                                                        "positivity_last_step", "status_last_step")}
        out["mixed_vs_fp64"] = res["mixed"]["value"] / res["fp64"]["value"]
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        if tet:   # a 24^3-box sample (82,944 cells) of the same blast
            m = 24
            xo, to, vo = synth.tet_mesh(m, box=box)
            so = O.Solver3(O.Mesh3.tets(xo, to, vo, np.full((len(to), 4), 1, dtype=np.int32)), b["deg"])
        else:     # the oracle holds ~15 KB of work arrays per cell: a 48^3 sample of the same blast
            m = 48
            so = O.Solver3(O.Mesh3(m, m, m, box, (1,) * 6), b["deg"])
        Qo = so.project_fn(synth.ic_blast3d(m, hw))
        so.step(Qo, cfl=b["cfl"])
        t0 = time.time()
        k = 30
        for _ in range(k):
            so.step(Qo, cfl=b["cfl"])
        dtc = time.time() - t0
        out["cpu_baseline"] = {"value": so.N * 5 * so.ML * k / dtc, "unit": UNIT, "cores": O.lib().orc_num_threads(),
                               "kind": "oracle", "sample": "%d steps of the same blast on %d cells (%d^3 boxes), %.1f s" % (k, so.N, m, dtc)}
    print(json.dumps(out))


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (every rank gets it): the timed
    region of the slowest replica."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed (each rank the same replica workload) per
    second of the slowest rank's timed region."""
    return world * units_per_rank / seconds


def time_steps(L, sol, Q, cfl, steps, flush):
    """K steps, each one replay of the solver's captured step graph on its
    stream, bracketed by CUDA events on that stream; the L2 is flushed (256 MB
    write) before each.  Returns the summed device time in ms."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.nvtx.range_push("timed")        # lets a profiler select the timed steps (ncu --nvtx-include timed/)
    for k in range(steps):
        flush.fill_(float(k))
        evs[k][0].record()
        L.lxw_run(sol, Q, 1, cfl)
        evs[k][1].record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs)


def smooth_l1_error(L, stream, mixed, net=None, tau=0.02):
    """L1 error of the cell-average density against the exact advected wave
    (32x32 periodic P2, CFL 0.1, all limiters on, run to t = 0.1 with the last
    step shortened to land on it).  The exact solution is projected with the
    library's own projection (8th-order rule)."""
    import torch
    w = WORKLOADS["smooth"]
    _, sol = build_workload(L, "smooth", stream, mixed)
    if net is not None:
        L.lxw_solver_set_mlp(sol, net, tau)
    Q = project(L, sol, w)
    steps, t, _ = L.lxw_run_to(sol, Q, 0.1, w["cfl"])      # the device lands the last step on t = 0.1
    xy = L.lxw_projection_points(sol)
    ex = synth.exact_smooth_density(xy[..., 0], xy[..., 1], t)
    prim = torch.from_numpy(np.stack(np.broadcast_arrays(ex, 1.0, 1.0, 1.0), axis=-1).copy()).cuda()
    Qe = torch.empty(sol.q64_shape, dtype=torch.float64, device="cuda")
    L.lxw_project(sol, prim, Qe)
    Qf = L.to_q64(sol, Q) if mixed else Q
    dr = Qf[:, 0, :] - Qe[:, 0, :]                              # density modes
    l1 = torch.abs(dr[:, 0]).mean().item()                      # cell averages (unit square, equal cells)
    # L2 of the DG density against the projected exact one: the basis is
    # orthonormal on each cell, so ||.||^2 = sum_i |T_i| sum_l dQ_il^2
    l2 = torch.sqrt((dr ** 2).sum(dim=1).mean()).item()
    return {"l1": l1, "l2": l2, "t": t, "steps": steps}


def locate(wc, pts):
    """Element of the half-resolution mesh wc (nc x nc squares, the masked
    step grid, or 2 nc^2 triangles with the same jitter rule) holding each
    point, and the point's reference coordinates there."""
    x0, x1, y0, y1 = wc.get("box", (0.0, 1.0, 0.0, 1.0))
    ncx, ncy = (wc["nx"], wc["ny"]) if wc["kind"] == "step" else (wc["n"], wc["n"])
    nc = ncx
    hx, hy = (x1 - x0) / ncx, (y1 - y0) / ncy
    x, y = pts[:, 0], pts[:, 1]
    ix = np.clip(np.floor((x - x0) / hx).astype(np.int64), 0, ncx - 1)
    iy = np.clip(np.floor((y - y0) / hy).astype(np.int64), 0, ncy - 1)
    if wc["kind"] == "disk":
        from scipy.spatial import Delaunay
        xy, tv = synth.disk_triangles(wc["n"])
        B = int(np.count_nonzero(np.abs(np.hypot(xy[:, 0], xy[:, 1]) - synth.SEDOV_RADIUS) < 1e-12))
        # points outside the coarse polygon (between its chords and the fine one's) move inside
        # its inscribed circle
        rin = synth.SEDOV_RADIUS * np.cos(np.pi / B) * (1.0 - 1e-9)
        rr = np.hypot(pts[:, 0], pts[:, 1])
        p = np.where((rr > rin)[:, None], pts * (rin / np.maximum(rr, 1e-300))[:, None], pts)
        tri = Delaunay(xy)
        ks = tri.find_simplex(p)
        assert np.all(ks >= 0), "a point outside the coarse disk mesh"
        # the mesh numbers the same triangles in another order: match vertex triples
        nv = np.int64(len(xy))

        def key(t):
            t = np.sort(t.astype(np.int64), axis=1)
            return (t[:, 0] * nv + t[:, 1]) * nv + t[:, 2]

        kt = key(tv)
        srt = np.argsort(kt)
        pos = np.searchsorted(kt[srt], key(tri.simplices[ks]))
        e = srt[pos]
        assert np.array_equal(kt[e], key(tri.simplices[ks])), "a simplex missing from the mesh"
        v0, v1, v2 = xy[tv[e, 0]], xy[tv[e, 1]], xy[tv[e, 2]]
        ax, ay, bx, by = v1[:, 0] - v0[:, 0], v1[:, 1] - v0[:, 1], v2[:, 0] - v0[:, 0], v2[:, 1] - v0[:, 1]
        det = ax * by - ay * bx
        px, py = p[:, 0] - v0[:, 0], p[:, 1] - v0[:, 1]
        return e, np.stack([(px * by - py * bx) / det, (ax * py - ay * px) / det], axis=1)
    if wc["kind"] in ("quad", "step"):
        ref = np.stack([2.0 * ((x - x0) / hx - ix) - 1.0, 2.0 * ((y - y0) / hy - iy) - 1.0], axis=1)
        cell = iy * ncx + ix
        if wc["kind"] == "quad":
            return cell, ref
        keep = synth.diffraction_mask(ncx, ncy).ravel()
        assert keep[cell].all(), "a point inside the step"
        return (np.cumsum(keep) - 1)[cell], ref
    xy, tv = synth.structured_triangles(nc, jitter=0.2, seed=20160129, box=(x0, x1, y0, y1))
    best = np.full(len(x), -1, dtype=np.int64)
    bmin = np.full(len(x), -np.inf)
    bref = np.zeros((len(x), 2))
    # vertices move by at most 0.2 h: the point lies in a triangle of the 3 x 3 squares around it
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            si, sj = ix + di, iy + dj
            ok = (si >= 0) & (si < nc) & (sj >= 0) & (sj < nc)
            for half in (0, 1):
                t = np.where(ok, 2 * (np.clip(sj, 0, nc - 1) * nc + np.clip(si, 0, nc - 1)) + half, 0)
                v0, v1, v2 = xy[tv[t, 0]], xy[tv[t, 1]], xy[tv[t, 2]]
                ax, ay, bx, by = v1[:, 0] - v0[:, 0], v1[:, 1] - v0[:, 1], v2[:, 0] - v0[:, 0], v2[:, 1] - v0[:, 1]
                det = ax * by - ay * bx
                px, py = x - v0[:, 0], y - v0[:, 1]
                xi = (px * by - py * bx) / det
                eta = (ax * py - ay * px) / det
                lm = np.minimum(np.minimum(xi, eta), 1.0 - xi - eta)
                upd = ok & (lm > bmin)
                best = np.where(upd, t, best); bmin = np.where(upd, lm, bmin)
                bref[upd] = np.stack([xi[upd], eta[upd]], axis=1)
    assert np.all(bmin > -1e-9), "a point outside the coarse mesh"
    return best, bref


def discretization_check(L, stream, name, net, tau, steps):
    """How 'equal' the errors are where no exact solution exists: the L1
    distance (density cell averages, area-weighted) of the mixed + learned
    result from the FP64 result at the same time, against the FP64 form's
    discretization-error estimate || u_N - P(u_{N/2}) ||_L1, P the L2
    projection of the half-resolution solution onto the fine elements."""
    import torch
    w = WORKLOADS[name]
    _, sf = build_workload(L, name, stream, False)
    Qf = project(L, sf, w)
    T = 0.0
    for _ in range(steps):
        T += L.lxw_step(sf, Qf, 0.0, w["cfl"], diag=True)["dt"]
    _, sm = build_workload(L, name, stream, True)
    L.lxw_solver_set_mlp(sm, net, tau)
    Qm = project(L, sm, w)
    km = L.lxw_run_to(sm, Qm, T, w["cfl"])[0]
    wc = half_resolution(w)
    _, sc = build_solver(L, wc, stream, False)
    Qc = project(L, sc, wc)
    kc = L.lxw_run_to(sc, Qc, T, w["cfl"])[0]
    # the coarse density at the fine projection points, projected onto the fine elements
    pts = L.lxw_projection_points(sf)
    N, npj = pts.shape[0], pts.shape[1]
    elem, ref = locate(wc, pts.reshape(-1, 2))
    phi = L.lxw_basis_eval(1 if w["kind"] in ("tri", "disk") else 0, w["deg"], ref)
    rc = np.einsum("pl,pl->p", Qc[:, 0, :].cpu().numpy()[elem], phi).reshape(N, npj)
    prim = np.stack([rc, np.zeros_like(rc), np.zeros_like(rc), np.ones_like(rc)], axis=-1)
    Qp = torch.zeros(sf.q64_shape, dtype=torch.float64, device="cuda")
    L.lxw_project(sf, torch.from_numpy(np.ascontiguousarray(prim)).cuda(), Qp)
    rho_f = Qf[:, 0, 0].cpu().numpy()
    rho_p = Qp[:, 0, 0].cpu().numpy()
    rho_m = L.to_q64(sm, Qm)[:, 0, 0].cpu().numpy()
    if w["kind"] not in ("tri", "disk"):
        area = np.full(N, 1.0 / N)
    else:
        xy, tv = (synth.disk_triangles(w["n"]) if w["kind"] == "disk"
                  else synth.structured_triangles(w["n"], jitter=0.2, seed=20160129))
        v0, v1, v2 = xy[tv[:, 0]], xy[tv[:, 1]], xy[tv[:, 2]]
        area = 0.5 * np.abs((v1[:, 0] - v0[:, 0]) * (v2[:, 1] - v0[:, 1]) - (v1[:, 1] - v0[:, 1]) * (v2[:, 0] - v0[:, 0]))
    e = float(np.sum(area * np.abs(rho_f - rho_p)))
    dist = float(np.sum(area * np.abs(rho_m - rho_f)))
    return {"t": T, "steps_fine": steps, "steps_mixed_learned": km, "steps_coarse": kc, "coarse_elements": sc.N,
            "l1_fp64_minus_projected_coarse": e, "l1_mixed_learned_minus_fp64": dist, "ratio": dist / e,
            "target_ratio_at_most": 0.1,
            "norm": "sum over fine elements of |T_i| |rho_avg difference| (density cell averages)"}



def fma_probes():
    """Measured FP64 / FP32 FMA-pipe throughput (TFLOP/s) from bench_fma_probe.cu,
    compiled next to this file on first use (a measurement aid of the bench,
    not part of the library); None where it cannot be built or run."""
    import ctypes
    import subprocess
    here = os.path.dirname(os.path.abspath(__file__))
    src, lib = os.path.join(here, "bench_fma_probe.cu"), os.path.join(here, "bench_fma_probe.so")
    try:
        if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            subprocess.run(["nvcc", "-O3", "-shared", "-Xcompiler", "-fPIC", "-gencode",
                            "arch=compute_103a,code=sm_103a", "-o", lib, src], check=True, capture_output=True)
        P = ctypes.CDLL(lib)
        P.fma_probe_tflops.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        out = {}
        for name, fp64 in (("fp64", 1), ("fp32", 0)):
            v = ctypes.c_double()
            out[name] = v.value if P.fma_probe_tflops(fp64, ctypes.byref(v)) == 0 else None
        return out
    except Exception:
        return {"fp64": None, "fp32": None}

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config5", choices=sorted(WORKLOADS) + sorted(CONFIGS) + ["ensemble", "blast3d", "blast3t"])
    ap.add_argument("--tau", type=float, default=0.01, help="learned gate: skip where theta_hat >= 1 - tau")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n3", type=int, default=0, help="blast3d / blast3t: cells (boxes) per axis instead of the default")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default work list of the mixed forms")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 100,352-triangle secondary line")
    ap.add_argument("--form", default="all", choices=["all", "learned", "mixed", "fp64"],
                    help="all: FP64, mixed and mixed + learned (headline); otherwise time only that form")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload in ("blast3d", "blast3t"):
        return run_blast3d(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1601_08145_gb300 import build, lxw as L
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    probes = fma_probes()

    def prepare(name, mixed, net):
        w, sol = build_workload(L, name, stream, mixed)
        if net is not None:
            L.lxw_solver_set_mlp(sol, net, args.tau)
        Q = project(L, sol, w)
        tune = None
        if mixed and not args.no_autotune:
            tune = L.lxw_autotune(sol, Q, w["cfl"], reps=3)     # on a scratch copy; Q is restored
        L.lxw_run(sol, Q, max(args.warmup, 3), w["cfl"])
        return dict(name=name, w=w, sol=sol, Q=Q, tune=tune, dof=sol.N * 4 * sol.ML)

    def timed_form(workload, mixed, clocks=None, net=None):
        """Every part of the workload prepared (solver, data, autotuned work
        list, warm-up), then K timed steps of each; the workload's time is the
        sum over its parts."""
        parts = [prepare(p, mixed, net) for p in parts_of(workload)]
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
            time.sleep(0.5)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for f in parts:
            f["total_ms"] = time_steps(L, f["sol"], f["Q"], f["w"]["cfl"], args.steps, flush)
        if world > 1:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        total_ms = sum(f["total_ms"] for f in parts)
        if world > 1:
            total_ms = max_over_ranks(total_ms, dist, "cuda")
        # per-phase device times from a separately traced pass (event nodes between the phases)
        for f in parts:
            ph = []
            for k in range(5):
                flush.fill_(float(k))
                ph.append(L.lxw_profile_step(f["sol"], f["Q"], f["w"]["cfl"]))
            f["phases"] = {k: statistics.mean(p[k] for p in ph) for k in ph[0]}
        dof = sum(f["dof"] for f in parts)
        phases = {k: sum(f["phases"][k] for f in parts) for k in parts[0]["phases"]}
        return dict(parts=parts, total_ms=total_ms, dof=dof, value=whole_job_rate(dof * args.steps, world, total_ms / 1e3),
                    phases=phases, clocks=clk, launches=sum(L.lxw_step_launches(f["sol"]) for f in parts))

    def e2e_of(form):
        """End to end through the public C ABI on HOST memory: every step, for
        every part, the host-to-device copy of the state (pinned, in the
        solver's own layout: the mixed form's packed FP64 averages + FP32
        modes), one step, the device-to-host copy of the result
        (lxw_run_host_state).  The FP64-layout entry (lxw_run_host: the state
        as Q[N][4][ML] doubles, converted on the way) is timed beside it."""
        def timed(fns):
            for fn in fns:
                fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                for fn in fns:
                    fn()
            return time.perf_counter() - t0
        state_fns, q64_fns, sbytes, qbytes = [], [], 0, 0
        for f in form["parts"]:
            sol, cfl = f["sol"], f["w"]["cfl"]
            Sh = torch.empty(sol.state_shape, dtype=torch.float64).pin_memory()
            Sh.copy_(f["Q"].cpu())
            Qh = torch.empty(sol.q64_shape, dtype=torch.float64).pin_memory()
            Qh.copy_((L.to_q64(sol, f["Q"]) if sol.mixed else f["Q"]).cpu())
            state_fns.append(lambda sol=sol, Sh=Sh, cfl=cfl: L.lxw_run_host_state(sol, Sh, 1, cfl))
            q64_fns.append(lambda sol=sol, Qh=Qh, cfl=cfl: L.lxw_run_host(sol, Qh, 1, cfl))
            sbytes += sol.state_bytes; qbytes += f["dof"] * 8
        e2e_s, q64_s = timed(state_fns), timed(q64_fns)
        dof = form["dof"]
        return {"value": world * dof * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": sbytes, "d2h_bytes_per_step": sbytes,
                "api": "lxw_run_host_state (host copy of the solver's state layout), every part every step",
                "fp64_layout": {"value": world * dof * args.steps / q64_s, "api": "lxw_run_host",
                                "h2d_bytes_per_step": qbytes, "d2h_bytes_per_step": qbytes}}

    def roofline_of(form, mixed):
        """The dominant kernel's roofline: the CK kernel (k_ck_mx on the FP32
        pipe, k_ck on the FP64 pipe); achieved = algorithmic flops of its
        launches over all parts / their summed CUDA-event time."""
        flops = sum(ck_flops_per_element(f["w"]["kind"], f["w"]["deg"]) * f["sol"].N for f in form["parts"])
        ck_ms = sum(f["phases"]["ck"] for f in form["parts"])
        ach = flops / (ck_ms / 1e3) / 1e12
        peak = FP32_PEAK_TFLOPS if mixed else FP64_PEAK_TFLOPS
        tr = [ck_traffic(f["name"], mixed, f["sol"].N) for f in form["parts"]]
        probe = probes["fp32" if mixed else "fp64"]
        return {"kernel": "k_ck_mx" if mixed else "k_ck", "dominant_phase": max(form["phases"], key=form["phases"].get),
                "bound": "alu", "pipe": "fp32" if mixed else "fp64", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": sum(tr) / len(tr) if all(t is not None for t in tr) else None,
                "traffic_per_part": dict(zip([f["name"] for f in form["parts"]], tr)),
                "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz" if mixed
                                else "nominal GB300 FP64 rate (recipe table)"),
                "peak_measured_fma_probe": probe, "frac_of_measured_probe": ach / probe if probe else None,
                "algorithmic_flops_per_launch": flops / len(form["parts"]),
                "launch_ms": ck_ms / len(form["parts"]),
                "per_part": {f["name"]: {"frac": ck_flops_per_element(f["w"]["kind"], f["w"]["deg"]) * f["sol"].N
                                         / (f["phases"]["ck"] / 1e3) / 1e12 / peak, "launch_ms": f["phases"]["ck"]}
                             for f in form["parts"]}}

    config = {"workload": desc_of(args.workload), "parts": {p: WORKLOADS[p]["desc"] for p in parts_of(args.workload)},
              "cfl": 0.1, "l2": "flushed between timed steps (256 MB write)",
              "timing": "one CUDA-graph replay per step and part, CUDA events on the solver's stream, summed over parts",
              "parallelism": "replicas" if world > 1 else "single GPU"}

    if args.form != "all":
        mixed = args.form != "fp64"
        net, info = train_indicator(L, stream, args.tau) if args.form == "learned" else (None, None)
        f = timed_form(args.workload, mixed, ClockSampler(local), net=net)
        e2e = e2e_of(f)
        if world > 1:
            dist.barrier()
        if rank == 0:
            out = {"metric": METRIC, "value": f["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                   "warmup": args.warmup, "ms_per_step": f["total_ms"] / args.steps, "higher_is_better": True,
                   "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64",
                   "data": "synthetic", "config": dict(config, elements=sum(x["sol"].N for x in f["parts"]),
                                                       dof_per_step=f["dof"], form=args.form),
                   "roofline": roofline_of(f, mixed), "e2e": e2e, "gpu_launches": args.steps * f["launches"],
                   "clocks": f["clocks"], "phases_ms": f["phases"],
                   "autotune": {x["name"]: x["tune"] for x in f["parts"]}, "learned_indicator": info}
            if world == 1 and not args.no_cpu_baseline:
                out["cpu_baseline"], _, _ = cpu_baseline(args.workload)
            print(json.dumps(out))
        if world > 1:
            dist.destroy_process_group()
        return

    fp64 = timed_form(args.workload, False)
    plain_mx = timed_form(args.workload, True)
    t_train = time.perf_counter()
    net, train_info = train_indicator(L, stream, args.tau)
    t_train = time.perf_counter() - t_train
    mx = timed_form(args.workload, True, ClockSampler(local), net=net)
    # one more (untimed) step per part with diagnostics: how often the FP64 paths ran and the gate skipped;
    # the other forms take the same step so that all three compare at the same time
    diags = {}
    for a, b, c in zip(mx["parts"], fp64["parts"], plain_mx["parts"]):
        diags[a["name"]] = L.lxw_step(a["sol"], a["Q"], 0.0, a["w"]["cfl"], diag=True)
        L.lxw_step(b["sol"], b["Q"], 0.0, b["w"]["cfl"])
        L.lxw_step(c["sol"], c["Q"], 0.0, c["w"]["cfl"])

    # distance of the mixed forms from the FP64 form after the same steps (density, relative L1), per part
    def l1_rel(form):
        out = {}
        for f, g in zip(form["parts"], fp64["parts"]):
            r = L.to_q64(f["sol"], f["Q"])[:, 0, 0]
            rf = g["Q"][:, 0, 0]
            out[f["name"]] = (torch.abs(r - rf).sum() / torch.abs(rf).sum()).item()
        return out
    dist_learned, dist_plain_mx = l1_rel(mx), l1_rel(plain_mx)
    # "at equal L1 error": the three forms against the exact smooth solution
    acc = {"fp64": smooth_l1_error(L, stream, False), "mixed": smooth_l1_error(L, stream, True),
           "mixed_learned": smooth_l1_error(L, stream, True, net=net, tau=args.tau)}
    acc["ratio_l1_mixed_learned_vs_fp64"] = acc["mixed_learned"]["l1"] / acc["fp64"]["l1"]
    acc["ratio_l2_mixed_learned_vs_fp64"] = acc["mixed_learned"]["l2"] / acc["fp64"]["l2"]
    acc["config"] = (WORKLOADS["smooth"]["desc"] + ", CFL 0.1, to t = 0.1; l1: cell-average density, "
                     "l2: DG density (all modes) against the projected exact solution")
    disc = {p: discretization_check(L, stream, p, net, args.tau, min(args.steps, 100))
            for p in parts_of(args.workload) if p != "smooth"}
    if disc:
        disc["ratio_max"] = max(d["ratio"] for d in disc.values())

    roofline = roofline_of(mx, True)
    plain = {"value": fp64["value"], "ms_per_step": fp64["total_ms"] / args.steps, "phases_ms": fp64["phases"],
             "roofline": roofline_of(fp64, False)}
    e2e = e2e_of(mx)

    # the 100,352-triangle rarefaction beside the headline (same network)
    secondary = None
    if not args.no_secondary and args.workload != "rarefy":
        s_mx = timed_form("rarefy", True, net=net)
        s_pm = timed_form("rarefy", True)
        s_64 = timed_form("rarefy", False)
        secondary = {"workload": WORKLOADS["rarefy"]["desc"], "value": s_mx["value"],
                     "ms_per_step": s_mx["total_ms"] / args.steps, "phases_ms": s_mx["phases"],
                     "roofline": roofline_of(s_mx, True),
                     "plain_mixed": {"value": s_pm["value"], "ms_per_step": s_pm["total_ms"] / args.steps},
                     "plain_fp64": {"value": s_64["value"], "ms_per_step": s_64["total_ms"] / args.steps},
                     "speedup_vs_plain_fp64": s_mx["value"] / s_64["value"],
                     "gain_vs_plain_mixed": s_mx["value"] / s_pm["value"]}
    if world > 1:
        dist.barrier()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    out = {"metric": METRIC, "value": mx["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": mx["total_ms"] / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": dict(config, elements=sum(f["sol"].N for f in mx["parts"]), dof_per_step=mx["dof"],
                          form="mixed + learned: FP32 bulk, FP64 averages/update/limiter solves, "
                               f"MLP-gated shock limiter (BF16 tensor-core inference, tau {args.tau})"),
           "roofline": roofline,
           "e2e": e2e,
           "gpu_launches": args.steps * mx["launches"],
           "clocks": mx["clocks"],
           "phases_ms": mx["phases"],
           "per_part": {f["name"]: {"ms_per_step": f["total_ms"] / args.steps, "phases_ms": f["phases"],
                                    "value": f["dof"] * args.steps / (f["total_ms"] / 1e3), "elements": f["sol"].N}
                        for f in mx["parts"]},
           "plain_fp64": plain,
           "speedup_vs_plain_fp64": mx["value"] / fp64["value"],
           "autotune": {f["name"]: f["tune"] for f in mx["parts"]},
           "plain_mixed": {"value": plain_mx["value"], "ms_per_step": plain_mx["total_ms"] / args.steps,
                           "phases_ms": plain_mx["phases"], "l1_rel_density_vs_fp64": dist_plain_mx,
                           "autotune": {f["name"]: f["tune"] for f in plain_mx["parts"]}},
           "learned_indicator": dict(train_info, train_s=t_train, tau=args.tau,
                                     skipped_cells_last_step={k: d["n_mlp_skip"] for k, d in diags.items()},
                                     gain_vs_plain_mixed=mx["value"] / plain_mx["value"]),
           "mixed_fp64_path_cells": {k: {"moment": d["n_fp64_moment"], "flux_limiter": d["n_fp64_edge"]}
                                     for k, d in diags.items()},
           "positivity_last_step": {k: {"min_rho": d["min_rho"], "min_p": d["min_p"]} for k, d in diags.items()},
           "l1_rel_density_vs_fp64": dist_learned,
           "smooth_l1_error": acc,
           "discretization_check": disc,
           "secondary": secondary}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"], _, _ = cpu_baseline(args.workload)
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
