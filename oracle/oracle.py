"""ctypes wrapper of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this module.  It marshals numpy arrays into the C oracle (lxw_oracle.c) and
holds none of the method's arithmetic.
"""
import contextlib
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

PERIODIC, REFLECT, TRANSPARENT, INFLOW = 0, 1, 2, 3
QUAD, TRI = 0, 1
DIAG_KEYS = ["s", "dt", "min_rho", "min_p", "mass", "momx", "momy", "energy",
             "n_mom", "n_edge", "n_sc", "status"]

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(C.CDLL(_build.build()))
    return _lib


@contextlib.contextmanager
def use_library(path):
    """Run this wrapper on another build of the oracle (a test's planted
    variant, same interface) inside the block."""
    global _lib
    keep = lib()
    _lib = _configure(C.CDLL(path))
    try:
        yield _lib
    finally:
        _lib = keep


def _configure(L):
    """Argument and result types of the oracle's C entry points."""
    L.orc_gauss_legendre.argtypes = [C.c_int, _dp, _dp]
    L.orc_num_modes.argtypes = [C.c_int, C.c_int]
    L.orc_basis_eval.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.orc_interior_rule.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
    for f in (L.orc_flux_d1, L.orc_flux_d2):
        f.argtypes = [C.c_double, _dp, _dp, _dp, _dp]
    L.orc_flux.argtypes = [C.c_double, _dp, _dp, _dp]
    L.orc_mesh_cartesian.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, _ip]
    L.orc_mesh_cartesian.restype = C.c_void_p
    L.orc_mesh_cartesian_masked.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                            _ip, C.POINTER(C.c_ubyte), C.c_int]
    L.orc_mesh_cartesian_masked.restype = C.c_void_p
    L.orc_solver_set_inflow.argtypes = [C.c_void_p, _dp]
    L.orc_mesh_triangles.argtypes = [C.c_int, _dp, C.c_int, _ip, _ip]
    L.orc_mesh_triangles.restype = C.c_void_p
    L.orc_mesh_free.argtypes = [C.c_void_p]
    for f in (L.orc_mesh_num_elements, L.orc_mesh_num_edges, L.orc_mesh_edges_per_element):
        f.argtypes = [C.c_void_p]
    L.orc_mesh_geometry.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
    L.orc_solver_new.argtypes = [C.c_void_p, C.c_int, C.c_double]
    L.orc_solver_new.restype = C.c_void_p
    L.orc_solver_free.argtypes = [C.c_void_p]
    L.orc_solver_set_params.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int]
    L.orc_solver_set_moment_exact.argtypes = [C.c_void_p, C.c_int]
    L.orc_solver_set_llf_global.argtypes = [C.c_void_p, C.c_int]
    L.orc_solver_set_ck_order.argtypes = [C.c_void_p, C.c_int]
    L.orc_flux_d3.argtypes = [C.c_double, _dp, _dp, _dp, _dp]
    L.orc_flux_d11.argtypes = [C.c_double, _dp, _dp, _dp, _dp, _dp]
    for f in (L.orc_solver_num_modes, L.orc_solver_num_points, L.orc_projection_num_points):
        f.argtypes = [C.c_void_p]
    L.orc_projection_points.argtypes = [C.c_void_p, _dp]
    L.orc_projection_weights.argtypes = [C.c_void_p, _dp]
    L.orc_project.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_eval_projection_points.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_eval_limiter_points.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_limiter_points.argtypes = [C.c_void_p, _dp]
    L.orc_last_fluxes.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_last_fluxes.restype = C.c_double
    L.orc_moment_limit.argtypes = [C.c_void_p, _dp, _dp, _ip]
    L.orc_moment_limit.restype = C.c_double
    L.orc_wave_speed.argtypes = [C.c_void_p, _dp]
    L.orc_wave_speed.restype = C.c_double
    L.orc_ck_element.argtypes = [C.c_void_p, _dp, C.c_int, C.c_double, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_mu_solve.argtypes = [C.c_double, C.c_double, _dp, _dp]
    L.orc_mu_solve.restype = C.c_double
    L.orc_flux_limit_cell.argtypes = [C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp]
    L.orc_shock_limit.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_step.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, _dp, _dp, _dp, _dp]
    L.orc_num_threads.argtypes = []
    L.orc_mlp_loss_grad.argtypes = [_dp, _dp, _dp, C.c_int, _dp, _dp]
    L.orc_mlp_loss_grad.restype = C.c_double
    L.orc_features.argtypes = [C.c_void_p, _dp, _dp]
    if hasattr(L, "orc3_step"):   # the 3D Cartesian oracle (a planted 2D variant may lack it)
        L.orc3_mode_exponents.argtypes = [C.c_int, _ip]
        L.orc3_basis_eval.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc3_flux.argtypes = [C.c_double, _dp, _dp]
        L.orc3_flux_series.argtypes = [C.c_double, C.c_int, _dp, _dp]
        L.orc3_mesh_cartesian.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _ip]
        L.orc3_mesh_cartesian.restype = C.c_void_p
        L.orc3_mesh_tets.argtypes = [C.c_int, _dp, C.c_int, _ip, _ip, _ip]
        L.orc3_mesh_tets.restype = C.c_void_p
        L.orc3_mesh_faces_per_element.argtypes = [C.c_void_p]
        L.orc3_tet_basis_eval.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc3_mesh_free.argtypes = [C.c_void_p]
        L.orc3_mesh_num_elements.argtypes = [C.c_void_p]
        L.orc3_mesh_geometry.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.orc3_solver_new.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.orc3_solver_new.restype = C.c_void_p
        L.orc3_solver_free.argtypes = [C.c_void_p]
        L.orc3_solver_set_params.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int]
        L.orc3_solver_set_llf_global.argtypes = [C.c_void_p, C.c_int]
        for f in (L.orc3_solver_num_modes, L.orc3_solver_num_points, L.orc3_projection_num_points):
            f.argtypes = [C.c_void_p]
        for f in (L.orc3_projection_points, L.orc3_projection_weights, L.orc3_limiter_points):
            f.argtypes = [C.c_void_p, _dp]
        for f in (L.orc3_project, L.orc3_eval_projection_points, L.orc3_eval_limiter_points):
            f.argtypes = [C.c_void_p, _dp, _dp]
        L.orc3_moment_limit.argtypes = [C.c_void_p, _dp, _dp, _ip]
        L.orc3_moment_limit.restype = C.c_double
        L.orc3_wave_speed.argtypes = [C.c_void_p, _dp]
        L.orc3_wave_speed.restype = C.c_double
        L.orc3_ck_element.argtypes = [C.c_void_p, _dp, C.c_int, C.c_double, _dp, _dp, _dp, _dp, _dp]
        L.orc3_flux_limit_cell.argtypes = [C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, _dp, _dp, _dp,
                                           _dp]
        L.orc3_mu_solve.argtypes = [C.c_double, C.c_double, _dp, _dp]
        L.orc3_mu_solve.restype = C.c_double
        L.orc3_shock_limit.argtypes = [C.c_void_p, _dp, _dp]
        L.orc3_step.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, _dp, _dp, _dp, _dp]
        L.orc3_last_fluxes.argtypes = [C.c_void_p, _dp, _dp]
        L.orc3_last_fluxes.restype = C.c_double
    return L


def gauss_legendre(n):
    x = np.zeros(n); w = np.zeros(n)
    lib().orc_gauss_legendre(n, _d(x), _d(w))
    return x, w


def interior_rule(kind, n):
    xi = np.zeros(n * n); eta = np.zeros(n * n); w = np.zeros(n * n)
    k = lib().orc_interior_rule(kind, n, _d(xi), _d(eta), _d(w))
    return xi[:k], eta[:k], w[:k]


def num_modes(kind, deg):
    return lib().orc_num_modes(kind, deg)


def basis_eval(kind, deg, xi, eta):
    xi = np.ascontiguousarray(xi, dtype=np.float64); eta = np.ascontiguousarray(eta, dtype=np.float64)
    ML = num_modes(kind, deg)
    phi = np.zeros((len(xi), ML)); dx = np.zeros_like(phi); dy = np.zeros_like(phi)
    lib().orc_basis_eval(kind, deg, len(xi), _d(xi), _d(eta), _d(phi), _d(dx), _d(dy))
    return phi, dx, dy


def flux(gamma, q):
    q = np.ascontiguousarray(q, dtype=np.float64); F = np.zeros(4); G = np.zeros(4)
    lib().orc_flux(gamma, _d(q), _d(F), _d(G))
    return F, G


def flux_d1(gamma, q, w):
    q = np.ascontiguousarray(q, dtype=np.float64); w = np.ascontiguousarray(w, dtype=np.float64)
    F = np.zeros(4); G = np.zeros(4)
    lib().orc_flux_d1(gamma, _d(q), _d(w), _d(F), _d(G))
    return F, G


def flux_d2(gamma, q, w):
    q = np.ascontiguousarray(q, dtype=np.float64); w = np.ascontiguousarray(w, dtype=np.float64)
    F = np.zeros(4); G = np.zeros(4)
    lib().orc_flux_d2(gamma, _d(q), _d(w), _d(F), _d(G))
    return F, G


def flux_d3(gamma, q, w):
    q = np.ascontiguousarray(q, dtype=np.float64); w = np.ascontiguousarray(w, dtype=np.float64)
    F = np.zeros(4); G = np.zeros(4)
    lib().orc_flux_d3(gamma, _d(q), _d(w), _d(F), _d(G))
    return F, G


def flux_d11(gamma, q, a, b):
    q = np.ascontiguousarray(q, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64); b = np.ascontiguousarray(b, dtype=np.float64)
    F = np.zeros(4); G = np.zeros(4)
    lib().orc_flux_d11(gamma, _d(q), _d(a), _d(b), _d(F), _d(G))
    return F, G


def mu_solve(gamma, eps0, qlxf, qc):
    a = np.ascontiguousarray(qlxf, dtype=np.float64); b = np.ascontiguousarray(qc, dtype=np.float64)
    return lib().orc_mu_solve(gamma, eps0, _d(a), _d(b))


def flux_limit_cell(gamma, eps0, area, dt, qbar, fW, fF):
    """Steps 4-5 of the flux limiter on one element; returns (proposals, cfl_bad)."""
    qbar = np.ascontiguousarray(qbar, dtype=np.float64)
    fW = np.ascontiguousarray(fW, dtype=np.float64); fF = np.ascontiguousarray(fF, dtype=np.float64)
    prop = np.zeros(fW.shape[0])
    bad = lib().orc_flux_limit_cell(gamma, eps0, fW.shape[0], area, dt, _d(qbar), _d(fW), _d(fF), _d(prop))
    return prop, bad


MLP_PARAMS = 24 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def mlp_loss_grad(P, X, y=None):
    """FP64 MLP: (loss, grad, yhat) on X[B][24] with targets y[B] (None: predictions only)."""
    P = np.ascontiguousarray(P, dtype=np.float64); X = np.ascontiguousarray(X, dtype=np.float64)
    B = X.shape[0]
    g = np.zeros(MLP_PARAMS); yh = np.zeros(B)
    yy = None if y is None else np.ascontiguousarray(y, dtype=np.float64)
    loss = lib().orc_mlp_loss_grad(_d(P), _d(X), _d(yy), B, _d(g) if y is not None else None, _d(yh))
    return loss, g, yh


def num_threads():
    return lib().orc_num_threads()


class Mesh:
    def __init__(self, ptr):
        if not ptr:
            raise ValueError("oracle mesh construction failed")
        self.ptr = ptr
        L = lib()
        self.N = L.orc_mesh_num_elements(ptr)
        self.E = L.orc_mesh_edges_per_element(ptr)
        self.nedges = L.orc_mesh_num_edges(ptr)

    @classmethod
    def cartesian(cls, nx, ny, box=(0.0, 1.0, 0.0, 1.0), bc=(PERIODIC,) * 4):
        b = np.array(bc, dtype=np.int32)
        return cls(lib().orc_mesh_cartesian(nx, ny, box[0], box[1], box[2], box[3], _i(b)))

    @classmethod
    def cartesian_masked(cls, nx, ny, box, bc, mask, mask_bc=1):
        """Cartesian mesh without the cells where mask[iy][ix] == 0."""
        b = np.array(bc, dtype=np.int32)
        mk = np.ascontiguousarray(mask, dtype=np.uint8).reshape(ny, nx)
        return cls(lib().orc_mesh_cartesian_masked(nx, ny, box[0], box[1], box[2], box[3], _i(b),
                                                   mk.ctypes.data_as(C.POINTER(C.c_ubyte)), mask_bc))

    @classmethod
    def triangles(cls, xy, tv, ebc=None):
        xy = np.ascontiguousarray(xy, dtype=np.float64); tv = np.ascontiguousarray(tv, dtype=np.int32)
        e = None if ebc is None else np.ascontiguousarray(ebc, dtype=np.int32)
        return cls(lib().orc_mesh_triangles(len(xy), _d(xy), len(tv), _i(tv), _i(e)))

    def geometry(self):
        a = np.zeros(self.N); p = np.zeros(self.N); cx = np.zeros(self.N); cy = np.zeros(self.N)
        lib().orc_mesh_geometry(self.ptr, _d(a), _d(p), _d(cx), _d(cy))
        return a, p, cx, cy

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.orc_mesh_free(self.ptr)
            self.ptr = None


class Solver:
    def __init__(self, mesh, deg, gamma=1.4, eps0=1e-12, alpha0=500.0, shock_limiter=True, moment_exact=False,
                 llf_global=False, ck_order=3):
        self.mesh = mesh  # keep alive
        self.ptr = lib().orc_solver_new(mesh.ptr, deg, gamma)
        if not self.ptr:
            raise ValueError("oracle solver construction failed")
        lib().orc_solver_set_params(self.ptr, eps0, alpha0, int(bool(shock_limiter)))
        lib().orc_solver_set_moment_exact(self.ptr, int(bool(moment_exact)))
        lib().orc_solver_set_llf_global(self.ptr, int(bool(llf_global)))
        if lib().orc_solver_set_ck_order(self.ptr, int(ck_order)):
            raise ValueError("ck_order must be 3 or 4")
        self.gamma = gamma
        self.N, self.E = mesh.N, mesh.E
        self.ML = lib().orc_solver_num_modes(self.ptr)
        self.npts = lib().orc_solver_num_points(self.ptr)
        self.nproj = lib().orc_projection_num_points(self.ptr)

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.orc_solver_free(self.ptr)
            self.ptr = None

    def set_inflow(self, prim):
        """State (rho, u, v, p) of the inflow boundaries."""
        lib().orc_solver_set_inflow(self.ptr, _d(np.ascontiguousarray(prim, dtype=np.float64)))

    def new_state(self):
        return np.zeros((self.N, 4, self.ML))

    def projection_points(self):
        xy = np.zeros((self.N, self.nproj, 2))
        lib().orc_projection_points(self.ptr, _d(xy))
        return xy

    def projection_weights(self):
        w = np.zeros(self.nproj)
        lib().orc_projection_weights(self.ptr, _d(w))
        return w

    def project(self, prim):
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        assert prim.shape == (self.N, self.nproj, 4)
        Q = self.new_state()
        lib().orc_project(self.ptr, _d(prim), _d(Q))
        return Q

    def project_fn(self, fn):
        """Project a primitive-variable function fn(x, y) -> (rho, u, v, p)."""
        xy = self.projection_points()
        r, u, v, p = fn(xy[..., 0], xy[..., 1])
        prim = np.stack(np.broadcast_arrays(r, u, v, p), axis=-1)
        return self.project(prim)

    def eval_projection_points(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        q = np.zeros((self.N, self.nproj, 4))
        lib().orc_eval_projection_points(self.ptr, _d(Q), _d(q))
        return q

    def eval_limiter_points(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        q = np.zeros((self.N, self.npts, 4))
        lib().orc_eval_limiter_points(self.ptr, _d(Q), _d(q))
        return q

    def limiter_points(self):
        xy = np.zeros((self.N, self.npts, 2))
        lib().orc_limiter_points(self.ptr, _d(xy))
        return xy

    def last_fluxes(self):
        """Outward f^LxW, f^LxF per element edge [N][E][4] and dt of the last step."""
        fw = np.zeros((self.N, self.E, 4)); ff = np.zeros((self.N, self.E, 4))
        dt = lib().orc_last_fluxes(self.ptr, _d(fw), _d(ff))
        return fw, ff, dt

    def moment_limit(self, Q):
        """In place; returns theta per element and the status bits."""
        th = np.zeros(self.N); st = C.c_int(0)
        lib().orc_moment_limit(self.ptr, _d(Q), _d(th), C.byref(st))
        return th, st.value

    def wave_speed(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        return lib().orc_wave_speed(self.ptr, _d(Q))

    def ck_element(self, Q, i, dt):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = [np.zeros((self.npts, 4)) for _ in range(5)]
        V = np.zeros((self.ML, 4))
        lib().orc_ck_element(self.ptr, _d(Q), i, dt, *[_d(o) for o in out], _d(V))
        return dict(q=out[0], qt=out[1], qtt=out[2], FT=out[3], GT=out[4], V=V)

    def features(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        F = np.zeros((self.N, 24))
        lib().orc_features(self.ptr, _d(Q), _d(F))
        return F

    def shock_limit(self, Q):
        th = np.zeros(self.N)
        lib().orc_shock_limit(self.ptr, _d(Q), _d(th))
        return th

    def step(self, Q, dt=0.0, cfl=0.1, want_theta=False):
        """Advance Q (in place) one step; returns the diagnostics dict."""
        assert Q.dtype == np.float64 and Q.flags.c_contiguous and Q.shape == (self.N, 4, self.ML)
        diag = np.zeros(16)
        tm = ts = te = None
        if want_theta:
            tm = np.zeros(self.N); ts = np.zeros(self.N); te = np.zeros((self.N, self.E))
        lib().orc_step(self.ptr, _d(Q), dt, cfl, _d(diag), _d(tm), _d(ts), _d(te))
        d = {k: diag[i] for i, k in enumerate(DIAG_KEYS)}
        d["status"] = int(d["status"])
        if want_theta:
            d.update(theta_mom=tm, theta_sc=ts, theta_edge=te)
        return d


# ---------------------------------------------------------------- 3D Cartesian
DIAG3_KEYS = ["s", "dt", "min_rho", "min_p", "mass", "momx", "momy", "momz", "energy",
              "n_mom", "n_face", "n_sc", "status"]


def mode_exponents3(deg):
    """(a, b, c) of each 3D mode, in the state's order."""
    n = (deg + 1) * (deg + 2) * (deg + 3) // 6
    abc = np.zeros(3 * n, dtype=np.int32)
    lib().orc3_mode_exponents(deg, _i(abc))
    return abc.reshape(n, 3)


def basis_eval3(deg, xi, eta, zeta, tet=False):
    """Hexahedral (tensor Legendre on [-1,1]^3) or tetrahedral basis and its
    reference gradient: [phi, d/dxi, d/deta, d/dzeta], each [npts][ML]."""
    xi, eta, zeta = (np.ascontiguousarray(a, dtype=np.float64) for a in (xi, eta, zeta))
    n = (deg + 1) * (deg + 2) * (deg + 3) // 6
    out = [np.zeros((len(xi), n)) for _ in range(4)]
    f = lib().orc3_tet_basis_eval if tet else lib().orc3_basis_eval
    f(deg, len(xi), _d(xi), _d(eta), _d(zeta), *[_d(o) for o in out])
    return out


def flux3(gamma, q):
    F = np.zeros((3, 5))
    lib().orc3_flux(gamma, _d(np.ascontiguousarray(q, dtype=np.float64)), _d(F))
    return F


def flux_series3(gamma, qs):
    """Taylor coefficients [K+1][3][5] of F(sum_k qs[k] t^k)."""
    qs = np.ascontiguousarray(qs, dtype=np.float64)
    Fs = np.zeros((qs.shape[0], 3, 5))
    lib().orc3_flux_series(gamma, qs.shape[0] - 1, _d(qs), _d(Fs))
    return Fs


def flux_limit_cell3(gamma, eps0, vol, dt, qbar, fW, fF):
    fW = np.ascontiguousarray(fW, dtype=np.float64); fF = np.ascontiguousarray(fF, dtype=np.float64)
    prop = np.zeros(fW.shape[0])
    bad = lib().orc3_flux_limit_cell(gamma, eps0, fW.shape[0], vol, dt,
                                     _d(np.ascontiguousarray(qbar, dtype=np.float64)), _d(fW), _d(fF), _d(prop))
    return prop, bad


class Mesh3:
    """Cartesian nx x ny x nz mesh of box = (x0, x1, y0, y1, z0, z1); bc per
    side (x-, x+, y-, y+, z-, z+): 0 periodic, 1 reflective, 2 transparent.
    Mesh3.tets(...) builds a tetrahedral mesh instead."""

    def __init__(self, nx, ny, nz, box=(0.0, 1.0, 0.0, 1.0, 0.0, 1.0), bc=(0,) * 6, _ptr=None):
        if _ptr is None:
            b = np.ascontiguousarray(box, dtype=np.float64)
            c = np.ascontiguousarray(bc, dtype=np.int32)
            _ptr = lib().orc3_mesh_cartesian(nx, ny, nz, _d(b), _i(c))
        if not _ptr:
            raise ValueError("oracle mesh construction failed")
        self.ptr = _ptr
        self.nx, self.ny, self.nz = nx, ny, nz
        self.N = lib().orc3_mesh_num_elements(self.ptr)
        self.E = lib().orc3_mesh_faces_per_element(self.ptr)

    @classmethod
    def tets(cls, xyz, tets, vid=None, fbc=None):
        """Tetrahedra xyz[nv][3], tets[nt][4], periodic vertex ids vid[nv]
        (None: the vertex index), boundary codes fbc[nt][4] of the faces
        opposite each vertex (None: transparent)."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        vid = np.ascontiguousarray(np.arange(len(xyz)) if vid is None else vid, dtype=np.int32)
        fb = None if fbc is None else np.ascontiguousarray(fbc, dtype=np.int32)
        ptr = lib().orc3_mesh_tets(len(xyz), _d(xyz), len(tets), _i(tets), _i(vid), _i(fb))
        return cls(0, 0, 0, _ptr=ptr)

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.orc3_mesh_free(self.ptr)
            self.ptr = None

    def geometry(self):
        vol, cx, cy, cz = (np.zeros(self.N) for _ in range(4))
        lib().orc3_mesh_geometry(self.ptr, _d(vol), _d(cx), _d(cy), _d(cz))
        return vol, cx, cy, cz


class Solver3:
    def __init__(self, mesh, deg, gamma=1.4, eps0=1e-12, alpha0=500.0, shock_limiter=True, llf_global=False):
        self.mesh = mesh
        self.ptr = lib().orc3_solver_new(mesh.ptr, deg, gamma)
        if not self.ptr:
            raise ValueError("oracle solver construction failed")
        lib().orc3_solver_set_params(self.ptr, eps0, alpha0, int(bool(shock_limiter)))
        lib().orc3_solver_set_llf_global(self.ptr, int(bool(llf_global)))
        self.gamma, self.deg, self.N = gamma, deg, mesh.N
        self.ML = lib().orc3_solver_num_modes(self.ptr)
        self.npts = lib().orc3_solver_num_points(self.ptr)
        self.nproj = lib().orc3_projection_num_points(self.ptr)

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.orc3_solver_free(self.ptr)
            self.ptr = None

    def new_state(self):
        return np.zeros((self.N, 5, self.ML))

    def projection_points(self):
        xyz = np.zeros((self.N, self.nproj, 3))
        lib().orc3_projection_points(self.ptr, _d(xyz))
        return xyz

    def projection_weights(self):
        w = np.zeros(self.nproj)
        lib().orc3_projection_weights(self.ptr, _d(w))
        return w

    def project(self, prim):
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        assert prim.shape == (self.N, self.nproj, 5)
        Q = self.new_state()
        lib().orc3_project(self.ptr, _d(prim), _d(Q))
        return Q

    def project_fn(self, fn):
        """Project fn(x, y, z) -> (rho, u, v, w, p)."""
        xyz = self.projection_points()
        vals = fn(xyz[..., 0], xyz[..., 1], xyz[..., 2])
        return self.project(np.stack(np.broadcast_arrays(*vals), axis=-1))

    def eval_projection_points(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        q = np.zeros((self.N, self.nproj, 5))
        lib().orc3_eval_projection_points(self.ptr, _d(Q), _d(q))
        return q

    def limiter_points(self):
        xyz = np.zeros((self.N, self.npts, 3))
        lib().orc3_limiter_points(self.ptr, _d(xyz))
        return xyz

    def eval_limiter_points(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        q = np.zeros((self.N, self.npts, 5))
        lib().orc3_eval_limiter_points(self.ptr, _d(Q), _d(q))
        return q

    def moment_limit(self, Q):
        th = np.zeros(self.N); st = C.c_int(0)
        lib().orc3_moment_limit(self.ptr, _d(Q), _d(th), C.byref(st))
        return th, st.value

    def wave_speed(self, Q):
        return lib().orc3_wave_speed(self.ptr, _d(np.ascontiguousarray(Q, dtype=np.float64)))

    def ck_element(self, Q, i, dt):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        q, qt, qtt = (np.zeros((self.npts, 5)) for _ in range(3))
        FT = np.zeros((self.npts, 3, 5)); V = np.zeros((self.ML, 5))
        lib().orc3_ck_element(self.ptr, _d(Q), i, dt, _d(q), _d(qt), _d(qtt), _d(FT), _d(V))
        return dict(q=q, qt=qt, qtt=qtt, FT=FT, V=V)

    def shock_limit(self, Q):
        th = np.zeros(self.N)
        lib().orc3_shock_limit(self.ptr, _d(Q), _d(th))
        return th

    def last_fluxes(self):
        E = self.mesh.E
        fw = np.zeros((self.N, E, 5)); ff = np.zeros((self.N, E, 5))
        dt = lib().orc3_last_fluxes(self.ptr, _d(fw), _d(ff))
        return fw, ff, dt

    def step(self, Q, dt=0.0, cfl=0.1, want_theta=False):
        assert Q.dtype == np.float64 and Q.flags.c_contiguous and Q.shape == (self.N, 5, self.ML)
        diag = np.zeros(16)
        tm = ts = tf = None
        if want_theta:
            tm = np.zeros(self.N); ts = np.zeros(self.N); tf = np.zeros((self.N, self.mesh.E))
        lib().orc3_step(self.ptr, _d(Q), dt, cfl, _d(diag), _d(tm), _d(ts), _d(tf))
        d = {k: diag[i] for i, k in enumerate(DIAG3_KEYS)}
        d["status"] = int(d["status"])
        if want_theta:
            d.update(theta_mom=tm, theta_sc=ts, theta_face=tf)
        return d
