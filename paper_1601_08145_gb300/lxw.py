"""Thin Python binding of the C ABI in include/lxw.h (ctypes).

Argument marshalling only: every step of the path runs in liblxw.so's CUDA
kernels.  Device buffers are torch CUDA tensors (float64, contiguous),
passed by data_ptr(); host buffers are numpy arrays.  Function names follow
the C entry points.  Importing works without a GPU; calling the library
needs liblxw.so built in-tree (``paper_1601_08145_gb300.build``) and fails
loudly when it is missing.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblxw.so")

OK, ERR_ARG, ERR_CUDA, ERR_NONPOSITIVE, ERR_CFL, ERR_NAN, ERR_BOUNDS, ERR_TIMEOUT, ERR_NOMEM = range(9)
BC_PERIODIC, BC_REFLECT, BC_TRANSPARENT, BC_INFLOW = 0, 1, 2, 3
KIND_QUAD, KIND_TRI = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
ST_NONPOSITIVE, ST_CFL, ST_NAN = 1, 2, 4

# every extern "C" symbol declared in include/lxw.h
EXPORTS = [
    "lxw_last_error", "lxw_options_default", "lxw_mesh_cartesian", "lxw_mesh_triangles",
    "lxw_mesh_destroy", "lxw_mesh_num_elements", "lxw_solver_create", "lxw_solver_destroy",
    "lxw_solver_set_stream", "lxw_solver_info", "lxw_projection_points", "lxw_project",
    "lxw_step", "lxw_run", "lxw_run_host", "lxw_moment_limit", "lxw_shock_limit",
    "lxw_step_launches", "lxw_profile_step", "lxw_step_phases", "lxw_workspace_copy",
    "lxw_moment_limit_noalloc", "lxw_state_bytes", "lxw_state_pack", "lxw_state_unpack",
    "lxw_batch_create", "lxw_batch_scalars", "lxw_autotune",
    "lxw_mlp_create", "lxw_mlp_destroy", "lxw_mlp_num_params", "lxw_mlp_get_params", "lxw_mlp_set_params",
    "lxw_mlp_forward", "lxw_mlp_loss_grad", "lxw_mlp_train", "lxw_solver_set_mlp", "lxw_step_dump",
    "lxw_step_gate", "lxw_profile_phases", "lxw_basis_eval", "lxw_mesh_cartesian_masked",
    "lxw_solver_set_inflow", "lxw_mlp_set_envelope", "lxw_mlp_get_envelope", "lxw_run_host_state",
    "lxw_solver_set_gate_wait_test", "lxw_run_to", "lxw_solver_get_options",
    "lxw3_solver_create", "lxw3_solver_destroy", "lxw3_solver_info", "lxw3_projection_points",
    "lxw3_project", "lxw3_step", "lxw3_run", "lxw3_profile_step", "lxw3_step_launches",
    "lxw3_solver_create_tets", "lxw3_faces_per_element",
]


class Options(C.Structure):
    _fields_ = [("gamma", C.c_double), ("eps0", C.c_double), ("alpha0", C.c_double),
                ("shock_limiter", C.c_int), ("precision", C.c_int), ("block_threads", C.c_int),
                ("ctas_per_sm", C.c_int), ("high_occupancy", C.c_int), ("moment_exact", C.c_int),
                ("llf_global", C.c_int), ("ck_order", C.c_int), ("gate_scan", C.c_int),
                ("reserved", C.c_int * 3)]


class Diag(C.Structure):
    _fields_ = [("s", C.c_double), ("dt", C.c_double), ("min_rho", C.c_double), ("min_p", C.c_double),
                ("mass", C.c_double), ("momx", C.c_double), ("momy", C.c_double), ("energy", C.c_double),
                ("n_mom", C.c_double), ("n_edge", C.c_double), ("n_sc", C.c_double),
                ("status", C.c_int), ("reserved", C.c_int),
                ("n_fp64_moment", C.c_double), ("n_fp64_edge", C.c_double), ("n_mlp_skip", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class LxwError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lxw status {code}: {msg}")
        self.code = code


_lib = None
_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def lib():
    """Load liblxw.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1601_08145_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    L.lxw_last_error.restype = C.c_char_p
    L.lxw_options_default.argtypes = [C.POINTER(Options)]
    L.lxw_mesh_cartesian.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, _ip, C.POINTER(_vp)]
    L.lxw_mesh_triangles.argtypes = [C.c_int, _dp, C.c_int, _ip, _ip, C.POINTER(_vp)]
    L.lxw_mesh_destroy.argtypes = [_vp]
    L.lxw_mesh_destroy.restype = None
    L.lxw_mesh_num_elements.argtypes = [_vp]
    L.lxw_solver_create.argtypes = [_vp, C.c_int, C.POINTER(Options), _vp, C.POINTER(_vp)]
    L.lxw_solver_destroy.argtypes = [_vp]
    L.lxw_solver_destroy.restype = None
    L.lxw_solver_set_stream.argtypes = [_vp, _vp]
    L.lxw_mesh_cartesian_masked.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, _ip,
                                            C.POINTER(C.c_ubyte), C.c_int, C.POINTER(_vp)]
    L.lxw_solver_set_inflow.argtypes = [_vp, _dp]
    L.lxw_solver_info.argtypes = [_vp, _ip, _ip, _ip, _ip, _ip]
    L.lxw_projection_points.argtypes = [_vp, _dp]
    L.lxw_project.argtypes = [_vp, _vp, _vp]
    L.lxw_step.argtypes = [_vp, _vp, C.c_double, C.c_double, C.POINTER(Diag), _vp, _vp]
    L.lxw_run.argtypes = [_vp, _vp, C.c_int, C.c_double, C.POINTER(Diag)]
    L.lxw_run_host.argtypes = [_vp, _vp, C.c_int, C.c_double, C.POINTER(Diag)]
    L.lxw_run_host_state.argtypes = [_vp, _vp, C.c_int, C.c_double, C.POINTER(Diag)]
    L.lxw_moment_limit.argtypes = [_vp, _vp, _vp, _vp]
    L.lxw_shock_limit.argtypes = [_vp, _vp, _vp]
    L.lxw_step_launches.argtypes = [_vp]
    L.lxw_profile_phases.argtypes = [_vp]
    L.lxw_basis_eval.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp]
    L.lxw_profile_step.argtypes = [_vp, _vp, C.c_double, C.POINTER(C.c_float)]
    L.lxw_step_phases.argtypes = [_vp, _vp, C.c_double, C.c_double, C.c_int]
    L.lxw_workspace_copy.argtypes = [_vp, C.c_int, _dp, C.c_size_t]
    L.lxw_batch_create.argtypes = [C.c_int, C.POINTER(_vp), C.c_int, C.POINTER(Options), _vp, C.POINTER(_vp)]
    L.lxw_batch_scalars.argtypes = [_vp, C.POINTER(C.c_int), _dp, _dp]
    L.lxw_autotune.argtypes = [_vp, _vp, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                               C.POINTER(C.c_float), C.POINTER(C.c_int)]
    L.lxw_mlp_create.argtypes = [C.c_int, C.c_ulonglong, _vp, C.POINTER(_vp)]
    L.lxw_mlp_destroy.argtypes = [_vp]
    L.lxw_mlp_destroy.restype = None
    L.lxw_mlp_num_params.argtypes = []
    L.lxw_mlp_get_params.argtypes = [_vp, _vp]
    L.lxw_mlp_set_params.argtypes = [_vp, _vp]
    L.lxw_mlp_forward.argtypes = [_vp, _vp, C.c_int, _vp]
    L.lxw_mlp_set_envelope.argtypes = [_vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]
    L.lxw_mlp_get_envelope.argtypes = [_vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]
    L.lxw_mlp_loss_grad.argtypes = [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_float), _vp]
    L.lxw_mlp_train.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, C.c_float, C.c_ulonglong,
                                C.POINTER(C.c_float)]
    L.lxw_solver_set_mlp.argtypes = [_vp, _vp, C.c_float]
    L.lxw_solver_set_gate_wait_test.argtypes = [_vp, C.c_longlong]
    L.lxw_solver_get_options.argtypes = [_vp, C.POINTER(Options)]
    L.lxw_run_to.argtypes = [_vp, _vp, C.c_double, C.c_double, C.c_int, _vp, C.POINTER(C.c_int), _dp]
    L.lxw_step_dump.argtypes = [_vp, _vp, C.c_double, _vp, _vp]
    L.lxw_step_gate.argtypes = [_vp, _vp, C.c_double, _vp, _vp]
    L.lxw_state_bytes.argtypes = [_vp]
    L.lxw_state_bytes.restype = C.c_size_t
    L.lxw_state_pack.argtypes = [_vp, _vp, _vp]
    L.lxw_state_unpack.argtypes = [_vp, _vp, _vp]
    L.lxw_moment_limit_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _vp, _vp, _vp, _vp, _vp]
    L.lxw3_solver_create.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _ip, C.c_int, C.POINTER(Options), _vp,
                                     C.POINTER(_vp)]
    L.lxw3_solver_destroy.argtypes = [_vp]
    L.lxw3_solver_destroy.restype = None
    L.lxw3_solver_info.argtypes = [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.lxw3_projection_points.argtypes = [_vp, _dp]
    L.lxw3_project.argtypes = [_vp, _vp, _vp]
    L.lxw3_step.argtypes = [_vp, _vp, C.c_double, C.c_double, _vp, _vp]
    L.lxw3_run.argtypes = [_vp, _vp, C.c_int, C.c_double, _vp]
    L.lxw3_profile_step.argtypes = [_vp, _vp, C.c_double, C.POINTER(C.c_float)]
    L.lxw3_step_launches.argtypes = [_vp]
    L.lxw3_solver_create_tets.argtypes = [C.c_int, _dp, C.c_int, _ip, _ip, _ip, C.c_int, C.POINTER(Options), _vp,
                                          C.POINTER(_vp)]
    L.lxw3_faces_per_element.argtypes = [_vp]
    _lib = L
    return L


def _check(st, allow=()):
    if st != OK and st not in allow:
        raise LxwError(st, lib().lxw_last_error().decode())
    return st


def _ptr(t, shape=None, what="tensor", torch_dtype="float64"):
    """data_ptr of a contiguous float64 (or int32) CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if torch_dtype == "int32":
        if not (t.is_cuda and not t.dtype.is_floating_point and t.element_size() == 4 and t.is_contiguous()):
            raise ValueError(f"{what}: need a contiguous int32 CUDA tensor")
    elif not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
        raise ValueError(f"{what}: need a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what}: shape {tuple(t.shape)} != {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def lxw_options_default(**kw):
    o = Options()
    _check(lib().lxw_options_default(C.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Mesh:
    def __init__(self, handle):
        self.h = handle
        self.N = lib().lxw_mesh_num_elements(handle)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lxw_mesh_destroy(self.h)
            self.h = None


def lxw_mesh_cartesian(nx, ny, box=(0.0, 1.0, 0.0, 1.0), bc=(BC_PERIODIC,) * 4):
    h = _vp()
    b = (C.c_int * 4)(*bc)
    _check(lib().lxw_mesh_cartesian(nx, ny, box[0], box[1], box[2], box[3], b, C.byref(h)))
    return Mesh(h)


def lxw_mesh_cartesian_masked(nx, ny, box, bc, mask, mask_bc=BC_REFLECT):
    """Cartesian grid without the cells where mask[iy][ix] == 0; faces towards
    those cells get mask_bc."""
    h = _vp()
    b = (C.c_int * 4)(*bc)
    mk = np.ascontiguousarray(mask, dtype=np.uint8).reshape(ny, nx)
    _check(lib().lxw_mesh_cartesian_masked(nx, ny, box[0], box[1], box[2], box[3], b,
                                           mk.ctypes.data_as(C.POINTER(C.c_ubyte)), mask_bc, C.byref(h)))
    return Mesh(h)


def lxw_mesh_triangles(xy, tv, ebc=None):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tv = np.ascontiguousarray(tv, dtype=np.int32)
    e = None if ebc is None else np.ascontiguousarray(ebc, dtype=np.int32)
    h = _vp()
    _check(lib().lxw_mesh_triangles(len(xy), xy.ctypes.data_as(_dp), len(tv), tv.ctypes.data_as(_ip),
                                    e.ctypes.data_as(_ip) if e is not None else None, C.byref(h)))
    return Mesh(h)


class Solver:
    def __init__(self, handle, mesh):
        self.h = handle
        self.mesh = mesh
        N, E, ML, npts, nproj = (C.c_int() for _ in range(5))
        _check(lib().lxw_solver_info(handle, C.byref(N), C.byref(E), C.byref(ML), C.byref(npts), C.byref(nproj)))
        self.N, self.E, self.ML, self.npts, self.nproj = N.value, E.value, ML.value, npts.value, nproj.value
        self.mq = 3 if self.ML == 6 else 4     # edge points per edge: degree + 1
        self.state_bytes = lib().lxw_state_bytes(handle)
        self.mixed = self.state_bytes != self.N * 4 * self.ML * 8
    @property
    def state_shape(self):
        """Shape of the float64 tensor holding the solver's state: Q[N][4][ML]
        for FP64 solvers, the packed bytes (as float64 words) for mixed ones."""
        return (self.state_bytes // 8,) if self.mixed else (self.N, 4, self.ML)

    @property
    def q64_shape(self):
        return (self.N, 4, self.ML)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lxw_solver_destroy(self.h)
            self.h = None


def lxw_solver_create(mesh, degree, options=None, stream=None):
    h = _vp()
    _check(lib().lxw_solver_create(mesh.h, degree, C.byref(options) if options is not None else None,
                                   _stream_handle(stream), C.byref(h)))
    return Solver(h, mesh)


def lxw_solver_set_stream(solver, stream):
    _check(lib().lxw_solver_set_stream(solver.h, _stream_handle(stream)))


def lxw_solver_set_inflow(solver, prim):
    """State (rho, u, v, p) of the solver's inflow faces."""
    p = np.ascontiguousarray(prim, dtype=np.float64)
    _check(lib().lxw_solver_set_inflow(solver.h, p.ctypes.data_as(_dp)))


def lxw_projection_points(solver):
    xy = np.zeros((solver.N, solver.nproj, 2))
    _check(lib().lxw_projection_points(solver.h, xy.ctypes.data_as(_dp)))
    return xy


def lxw_basis_eval(kind, degree, ref_xy):
    """Basis values [n][ML] at reference points ref_xy[n][2] (host, numpy)."""
    ref = np.ascontiguousarray(ref_xy, dtype=np.float64).reshape(-1, 2)
    ML = (degree + 1) * (degree + 2) // 2
    out = np.zeros((ref.shape[0], ML))
    _check(lib().lxw_basis_eval(kind, degree, ref.shape[0], ref.ctypes.data_as(_dp), out.ctypes.data_as(_dp)))
    return out


def lxw_project(solver, prim, Q):
    """Projection into Q64[N][4][ML] (pack it for mixed solvers)."""
    _check(lib().lxw_project(solver.h, _ptr(prim, (solver.N, solver.nproj, 4), "prim"),
                             _ptr(Q, solver.q64_shape, "Q")))


def lxw_state_pack(solver, Q64, state):
    _check(lib().lxw_state_pack(solver.h, _ptr(Q64, solver.q64_shape, "Q64"), _ptr(state, solver.state_shape, "state")))


def lxw_state_unpack(solver, state, Q64):
    _check(lib().lxw_state_unpack(solver.h, _ptr(state, solver.state_shape, "state"), _ptr(Q64, solver.q64_shape, "Q64")))


def new_state(solver, Q64=None):
    """A device state tensor for the solver, optionally packed from Q64."""
    import torch
    st = torch.zeros(solver.state_shape, dtype=torch.float64, device="cuda")
    if Q64 is not None:
        lxw_state_pack(solver, Q64, st)
    return st


def to_q64(solver, state):
    import torch
    if not solver.mixed:
        return state
    Q = torch.empty(solver.q64_shape, dtype=torch.float64, device="cuda")
    lxw_state_unpack(solver, state, Q)
    return Q


def _diag_result(st, d):
    out = d.as_dict()
    out["return_status"] = st
    return out


def lxw_step(solver, Q, dt=0.0, cfl=0.1, diag=False, theta_cell=None, theta_edge=None):
    d = Diag() if diag else None
    st = _check(lib().lxw_step(solver.h, _ptr(Q, solver.state_shape, "Q"), dt, cfl,
                               C.byref(d) if d is not None else None,
                               _ptr(theta_cell, (2, solver.N), "theta_cell"),
                               _ptr(theta_edge, (solver.N, solver.E), "theta_edge")),
                allow=(ERR_NONPOSITIVE, ERR_CFL, ERR_NAN, ERR_TIMEOUT))
    return _diag_result(st, d) if d is not None else None


def lxw_run(solver, Q, nsteps, cfl, diag=False):
    d = Diag() if diag else None
    st = _check(lib().lxw_run(solver.h, _ptr(Q, solver.state_shape, "Q"), nsteps, cfl,
                              C.byref(d) if d is not None else None), allow=(ERR_NONPOSITIVE, ERR_CFL, ERR_NAN, ERR_TIMEOUT))
    return _diag_result(st, d) if d is not None else None


def lxw_run_to(solver, Q, t_span, cfl, max_steps=10_000_000, diag=False):
    """Steps until the state has advanced by exactly t_span (the device
    shortens the last step); returns (steps, t_reached, diag dict or None)."""
    d = Diag() if diag else None
    k = C.c_int(0); t = C.c_double(0.0)
    st = _check(lib().lxw_run_to(solver.h, _ptr(Q, solver.state_shape, "Q"), t_span, cfl, max_steps,
                                 C.byref(d) if d is not None else None, C.byref(k), C.byref(t)),
                allow=(ERR_NONPOSITIVE, ERR_CFL, ERR_NAN, ERR_TIMEOUT))
    return k.value, t.value, (_diag_result(st, d) if d is not None else None)


def lxw_run_host(solver, Qh, nsteps, cfl, diag=False):
    """Qh: host buffer (numpy float64 array or pinned CPU torch tensor) [N][4][ML]."""
    if isinstance(Qh, np.ndarray):
        assert Qh.dtype == np.float64 and Qh.flags.c_contiguous and Qh.shape == solver.q64_shape
        p = C.c_void_p(Qh.ctypes.data)
    else:
        assert (not Qh.is_cuda) and Qh.element_size() == 8 and Qh.is_contiguous() and tuple(Qh.shape) == solver.q64_shape
        p = C.c_void_p(Qh.data_ptr())
    d = Diag() if diag else None
    st = _check(lib().lxw_run_host(solver.h, p, nsteps, cfl, C.byref(d) if d is not None else None),
                allow=(ERR_NONPOSITIVE, ERR_CFL, ERR_NAN, ERR_TIMEOUT))
    return _diag_result(st, d) if d is not None else None


def lxw_run_host_state(solver, Sh, nsteps, cfl, diag=False):
    """Sh: CPU torch tensor (pinned for DMA) holding the solver's state layout
    (float64 words, shape solver.state_shape)."""
    assert (not Sh.is_cuda) and Sh.element_size() == 8 and Sh.is_contiguous() and tuple(Sh.shape) == solver.state_shape
    d = Diag() if diag else None
    st = _check(lib().lxw_run_host_state(solver.h, C.c_void_p(Sh.data_ptr()), nsteps, cfl,
                                         C.byref(d) if d is not None else None),
                allow=(ERR_NONPOSITIVE, ERR_CFL, ERR_NAN, ERR_TIMEOUT))
    return _diag_result(st, d) if d is not None else None


def lxw_moment_limit(solver, Q, theta=None, s_out=None):
    _check(lib().lxw_moment_limit(solver.h, _ptr(Q, solver.state_shape, "Q"), _ptr(theta, (solver.N,), "theta"),
                                  _ptr(s_out, (1,), "s_out")))


def lxw_shock_limit(solver, Q, theta=None):
    _check(lib().lxw_shock_limit(solver.h, _ptr(Q, solver.state_shape, "Q"), _ptr(theta, (solver.N,), "theta")))


def lxw_step_launches(solver):
    return lib().lxw_step_launches(solver.h)


PHASES = ["reset", "moment", "ck", "edge", "update", "shock"]
PHASES_MIXED = ["moment", "ck", "edge", "update", "shock"]


def lxw_profile_phases(solver):
    return lib().lxw_profile_phases(solver.h)


def lxw_profile_step(solver, Q, cfl):
    """One step with CUDA-event timing of each phase; returns {phase: ms}."""
    n = lxw_profile_phases(solver)
    ms = (C.c_float * n)()
    _check(lib().lxw_profile_step(solver.h, _ptr(Q, solver.state_shape, "Q"), cfl, ms))
    names = PHASES_MIXED if solver.mixed else PHASES
    return {names[k]: float(ms[k]) for k in range(n)}


def lxw_step_phases(solver, Q, dt, cfl, nphases):
    _check(lib().lxw_step_phases(solver.h, _ptr(Q, solver.state_shape, "Q"), dt, cfl, nphases))


def lxw_workspace_copy(solver, which):
    """Workspace buffer after lxw_step_phases: 0 traces [E][MQ][8][N],
    1 fluxes [E][8][N], 2 proposals [E][N], 3 (s, dt)."""
    shapes = {0: (solver.E, solver.mq, 8, solver.N), 1: (solver.E, 8, solver.N), 2: (solver.E, solver.N), 3: (2,)}
    out = np.zeros(shapes[which])
    _check(lib().lxw_workspace_copy(solver.h, which, out.ctypes.data_as(_dp), out.size))
    return out


def lxw_moment_limit_noalloc(kind, degree, Q, theta=None, s_out=None, gamma=1.4, eps0=1e-12, stream=None,
                             status=None):
    """Allocation-free moment limiter + wave speed (no solver needed).
    Q: [N][4][ML] float64 CUDA tensor (ML of the kind and degree), in place;
    theta [N], s_out [1] float64; status [1] int32 (nullable: then the call
    waits and raises LxwError(ERR_NONPOSITIVE) for a non-positive average)."""
    if degree not in (2, 3) or kind not in (KIND_QUAD, KIND_TRI):
        raise LxwError(ERR_ARG, "lxw_moment_limit_noalloc: kind must be quad/triangle and degree 2 or 3")
    ML = (degree + 1) * (degree + 2) // 2
    if Q.dim() != 3 or Q.shape[1] != 4 or Q.shape[2] != ML:
        raise LxwError(ERR_ARG, "lxw_moment_limit_noalloc: Q must be [N][4][%d] for degree %d, got %s"
                       % (ML, degree, tuple(Q.shape)))
    N = Q.shape[0]
    _check(lib().lxw_moment_limit_noalloc(kind, degree, N, gamma, eps0, _ptr(Q, (N, 4, ML), "Q"),
                                          _ptr(theta, (N,), "theta"), _ptr(s_out, (1,), "s_out"),
                                          _ptr(status, (1,), "status", torch_dtype="int32"),
                                          _stream_handle(stream)))


def lxw_batch_create(meshes, degree, options=None, stream=None):
    """One solver over the disjoint union of independent problems."""
    arr = (_vp * len(meshes))(*[m.h for m in meshes])
    h = _vp()
    _check(lib().lxw_batch_create(len(meshes), arr, degree, C.byref(options) if options is not None else None,
                                  _stream_handle(stream), C.byref(h)))
    sol = Solver(h, list(meshes))
    sol.offsets = np.cumsum([0] + [m.N for m in meshes])
    return sol


def lxw_batch_scalars(solver):
    n = C.c_int()
    _check(lib().lxw_batch_scalars(solver.h, C.byref(n), None, None))
    sv = np.zeros(n.value); dv = np.zeros(n.value)
    _check(lib().lxw_batch_scalars(solver.h, C.byref(n), sv.ctypes.data_as(_dp), dv.ctypes.data_as(_dp)))
    return sv, dv


def lxw_autotune(solver, state, cfl, reps=5):
    b = C.c_int(); c = C.c_int(); ms = C.c_float(); hi = C.c_int()
    _check(lib().lxw_autotune(solver.h, _ptr(state, solver.state_shape, "state"), cfl, reps,
                              C.byref(b), C.byref(c), C.byref(ms), C.byref(hi)))
    return {"block_threads": b.value, "ctas_per_sm": c.value, "high_occupancy": hi.value,
            "gate_scan": lxw_solver_get_options(solver)["gate_scan"], "ms_per_step": ms.value}


def lxw_solver_get_options(solver):
    """The solver's options as it runs now (after lxw_autotune: its choices)."""
    o = Options()
    _check(lib().lxw_solver_get_options(solver.h, C.byref(o)))
    return {k: getattr(o, k) for k, _ in Options._fields_ if k != "reserved"}


MLP_IN, MLP_HIDDEN, MLP_PARAMS = 24, 64, 5825


def _fptr(t, shape=None, what="tensor"):
    """data_ptr of a contiguous float32 CUDA tensor."""
    if t is None:
        return None
    if not (t.is_cuda and t.element_size() == 4 and t.dtype.is_floating_point and t.is_contiguous()):
        raise ValueError(f"{what}: need a contiguous float32 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what}: shape {tuple(t.shape)} != {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


class Mlp:
    def __init__(self, h, max_batch):
        self.h = h
        self.max_batch = max_batch

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lxw_mlp_destroy(self.h)
            self.h = None


def lxw_mlp_create(max_batch, seed=1, stream=None):
    h = _vp()
    _check(lib().lxw_mlp_create(max_batch, seed, _stream_handle(stream), C.byref(h)))
    return Mlp(h, max_batch)


def lxw_mlp_num_params():
    return lib().lxw_mlp_num_params()


def lxw_mlp_get_params(mlp):
    import torch
    P = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    _check(lib().lxw_mlp_get_params(mlp.h, _fptr(P)))
    return P


def lxw_mlp_set_params(mlp, P):
    _check(lib().lxw_mlp_set_params(mlp.h, _fptr(P, (MLP_PARAMS,), "params")))


def lxw_mlp_forward(mlp, X):
    import torch
    y = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    _check(lib().lxw_mlp_forward(mlp.h, _fptr(X, (X.shape[0], MLP_IN), "X"), X.shape[0], _fptr(y)))
    return y


def lxw_mlp_loss_grad(mlp, X, y):
    import torch
    g = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = C.c_float()
    _check(lib().lxw_mlp_loss_grad(mlp.h, _fptr(X, (X.shape[0], MLP_IN), "X"), _fptr(y, (X.shape[0],), "y"),
                                   X.shape[0], C.byref(loss), _fptr(g)))
    return loss.value, g


def lxw_mlp_train(mlp, X, y, epochs, batch, lr, seed=7):
    loss = C.c_float()
    _check(lib().lxw_mlp_train(mlp.h, _fptr(X, (X.shape[0], MLP_IN), "X"), _fptr(y, (X.shape[0],), "y"), X.shape[0],
                               epochs, batch, lr, seed, C.byref(loss)))
    return loss.value


def lxw_mlp_set_envelope(mlp, lo=None, hi=None):
    """Per-feature bounds inside which the gate uses the network (None, None: unbounded)."""
    if lo is None or hi is None:
        _check(lib().lxw_mlp_set_envelope(mlp.h, None, None))
        return
    l = np.ascontiguousarray(lo, dtype=np.float32); h = np.ascontiguousarray(hi, dtype=np.float32)
    assert l.shape == h.shape == (MLP_IN,)
    _check(lib().lxw_mlp_set_envelope(mlp.h, l.ctypes.data_as(C.POINTER(C.c_float)), h.ctypes.data_as(C.POINTER(C.c_float))))


def lxw_mlp_get_envelope(mlp):
    l = np.zeros(MLP_IN, np.float32); h = np.zeros(MLP_IN, np.float32)
    _check(lib().lxw_mlp_get_envelope(mlp.h, l.ctypes.data_as(C.POINTER(C.c_float)), h.ctypes.data_as(C.POINTER(C.c_float))))
    return l, h


def lxw_solver_set_gate_wait_test(solver, cycles):
    """Test aid: > 0 makes the gated shock kernel's first wait expire after
    that many SM cycles (a barrier nothing arrives at); 0 switches it off."""
    _check(lib().lxw_solver_set_gate_wait_test(solver.h, int(cycles)))


def lxw_solver_set_mlp(solver, mlp, tau=0.05):
    _check(lib().lxw_solver_set_mlp(solver.h, mlp.h if mlp is not None else None, tau))


def lxw_step_dump(solver, state, cfl):
    """One mixed step; returns (features [N][24] float32, theta_sc [N] float64) of its shock limiter."""
    import torch
    F = torch.empty((solver.N, MLP_IN), dtype=torch.float32, device="cuda")
    th = torch.empty(solver.N, dtype=torch.float64, device="cuda")
    _check(lib().lxw_step_dump(solver.h, _ptr(state, solver.state_shape, "state"), cfl, _fptr(F), _ptr(th)))
    return F, th


def lxw_step_gate(solver, state, cfl, features=False):
    """One step gated by the solver's network; returns theta_hat [N] float32
    (NaN where the network was not asked) and, with features=True, the
    features [N][24] it saw."""
    import torch
    g = torch.empty(solver.N, dtype=torch.float32, device="cuda")
    F = torch.empty((solver.N, MLP_IN), dtype=torch.float32, device="cuda") if features else None
    _check(lib().lxw_step_gate(solver.h, _ptr(state, solver.state_shape, "state"), cfl, _fptr(g), _fptr(F)))
    return (g, F) if features else g


# ---------------------------------------------------------------- 3D Cartesian (FP64)
class Diag3(C.Structure):
    _fields_ = [("s", C.c_double), ("dt", C.c_double), ("min_rho", C.c_double), ("min_p", C.c_double),
                ("mass", C.c_double), ("momx", C.c_double), ("momy", C.c_double), ("momz", C.c_double),
                ("energy", C.c_double), ("n_mom", C.c_double), ("n_face", C.c_double), ("n_sc", C.c_double),
                ("status", C.c_int), ("reserved", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


PHASES3 = ("moment", "ck", "face", "update", "shock")


class Solver3:
    def __init__(self, handle, n3=None):
        self.h = handle
        self.nx, self.ny, self.nz = n3 if n3 is not None else (None, None, None)
        N, ML, nproj = (C.c_int() for _ in range(3))
        _check(lib().lxw3_solver_info(handle, C.byref(N), C.byref(ML), C.byref(nproj)))
        self.N, self.ML, self.nproj = N.value, ML.value, nproj.value
        self.E = lib().lxw3_faces_per_element(handle)

    @property
    def state_shape(self):
        return (self.N, 5, self.ML)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lxw3_solver_destroy(self.h)
            self.h = None


def lxw3_solver_create(nx, ny, nz, box, bc, degree, options=None, stream=None):
    """3D Cartesian FP64 solver: box = (x0, x1, y0, y1, z0, z1), bc per side (x-, x+, y-, y+, z-, z+)."""
    h = _vp()
    b = np.ascontiguousarray(box, dtype=np.float64)
    c = np.ascontiguousarray(bc, dtype=np.int32)
    _check(lib().lxw3_solver_create(nx, ny, nz, b.ctypes.data_as(_dp), c.ctypes.data_as(_ip), degree,
                                    C.byref(options) if options is not None else None, _stream_handle(stream),
                                    C.byref(h)))
    return Solver3(h, (nx, ny, nz))


def lxw3_solver_create_tets(xyz, tets, vid, degree, face_bc=None, options=None, stream=None):
    """3D tetrahedral FP64 solver from host arrays: vertex positions xyz[nv][3],
    positively oriented cells tets[nt][4], vertex ids vid[nv] (equal ids glue
    periodic faces), face_bc[nt][4] codes of unmatched faces (None: transparent)."""
    h = _vp()
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    v = np.ascontiguousarray(vid, dtype=np.int32).reshape(-1)
    if v.shape[0] != x.shape[0]:
        raise ValueError("vid needs one id per vertex")
    fb = None
    if face_bc is not None:
        fb = np.ascontiguousarray(face_bc, dtype=np.int32).reshape(-1, 4)
        if fb.shape[0] != t.shape[0]:
            raise ValueError("face_bc needs four codes per cell")
    _check(lib().lxw3_solver_create_tets(x.shape[0], x.ctypes.data_as(_dp), t.shape[0], t.ctypes.data_as(_ip),
                                         v.ctypes.data_as(_ip), fb.ctypes.data_as(_ip) if fb is not None else None,
                                         degree, C.byref(options) if options is not None else None,
                                         _stream_handle(stream), C.byref(h)))
    return Solver3(h)


def lxw3_projection_points(solver):
    xyz = np.zeros((solver.N, solver.nproj, 3))
    _check(lib().lxw3_projection_points(solver.h, xyz.ctypes.data_as(_dp)))
    return xyz


def lxw3_project(solver, prim, Q):
    _check(lib().lxw3_project(solver.h, _ptr(prim, (solver.N, solver.nproj, 5), "prim"),
                              _ptr(Q, solver.state_shape, "Q")))


def lxw3_step(solver, Q, dt=0.0, cfl=0.1, diag=False, theta_face=None):
    d = Diag3()
    st = _check(lib().lxw3_step(solver.h, _ptr(Q, solver.state_shape, "Q"), dt, cfl, C.byref(d),
                                _ptr(theta_face, (solver.N, solver.E), "theta_face")),
                allow=(ERR_NONPOSITIVE, ERR_CFL, ERR_NAN))
    return _diag_result(st, d) if diag else None


def lxw3_run(solver, Q, nsteps, cfl, diag=False):
    d = Diag3()
    st = _check(lib().lxw3_run(solver.h, _ptr(Q, solver.state_shape, "Q"), nsteps, cfl, C.byref(d)),
                allow=(ERR_NONPOSITIVE, ERR_CFL, ERR_NAN))
    return _diag_result(st, d) if diag else None


def lxw3_profile_step(solver, Q, cfl):
    ms = (C.c_float * 5)()
    _check(lib().lxw3_profile_step(solver.h, _ptr(Q, solver.state_shape, "Q"), cfl, ms))
    return {PHASES3[k]: float(ms[k]) for k in range(5)}


def lxw3_step_launches(solver):
    return lib().lxw3_step_launches(solver.h)
