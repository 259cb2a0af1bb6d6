"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.

This module holds problem data only -- meshes (vertex coordinates and
connectivity), initial conditions as primitive-variable point functions, and
seeded random states -- and none of the method's arithmetic (no basis,
quadrature, flux, limiter or geometry).  Each side (the CPU oracle and the
GPU library) builds its own geometry, tables and projections from these.

Workloads (the paper's Sec. 4 problems and the scaled synthetic cases built
from them):
  smooth   32x32 periodic [0,1]^2, rho = 1 + 0.2 sin 2pi(x+y), u = (1,1), p = 1
  rarefy   224x224x2 jittered triangles on [0,1]^2, rho = 1, p = 0.4,
           u = -2 (x < 0.5) / +2 (x > 0.5), transparent boundaries
  blast    1024x1024 on [-1.1,1.1]^2, rho = 1, u = 0, p = 1e-12 except the 4
           centre cells with E = 0.244816 / cell area, reflective walls
  paper_smooth  the Table 1 problem rho = 1 - 0.9999 sin 2pi x sin 2pi y,
           u = (1,0), p = 1, periodic
"""
import numpy as np

PERIODIC, REFLECT, TRANSPARENT = 0, 1, 2
GAMMA = 1.4
MASK64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n outputs of the SplitMix64 generator (Steele, Lea & Flood 2014)."""
    out = np.empty(n, dtype=np.uint64)
    x = seed & MASK64
    for i in range(n):
        x = (x + 0x9E3779B97F4A7C15) & MASK64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        out[i] = z ^ (z >> 31)
    return out


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0,1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def structured_triangles(n: int, jitter: float = 0.2, seed: int = 20160129,
                         box=(0.0, 1.0, 0.0, 1.0)):
    """n x n squares, each split by its '/' diagonal into two CCW triangles.

    Interior vertices move by U[-jitter, jitter] * h in each coordinate;
    boundary vertices move only along their side; corners stay fixed.
    Returns (xy[nv,2], tv[nt,3]).
    """
    x0, x1, y0, y1 = box
    hx, hy = (x1 - x0) / n, (y1 - y0) / n
    I, J = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    X = x0 + I * hx
    Y = y0 + J * hy
    if jitter > 0.0:
        r = uniform01(seed, 2 * (n + 1) * (n + 1)).reshape(2, n + 1, n + 1)
        dx = (2.0 * r[0] - 1.0) * jitter * hx
        dy = (2.0 * r[1] - 1.0) * jitter * hy
        onx = (I == 0) | (I == n)     # on a vertical side: x fixed
        ony = (J == 0) | (J == n)     # on a horizontal side: y fixed
        X = X + np.where(onx, 0.0, dx)
        Y = Y + np.where(ony, 0.0, dy)
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    vid = lambda i, j: j * (n + 1) + i
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    i = i.ravel(); j = j.ravel()
    a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
    t1 = np.stack([a, b, c], axis=1)
    t2 = np.stack([a, c, d], axis=1)
    tv = np.empty((2 * n * n, 3), dtype=np.int32)
    tv[0::2] = t1
    tv[1::2] = t2
    return xy, tv


# ---------------------------------------------------------------- initial data
def ic_smooth(x, y):
    return 1.0 + 0.2 * np.sin(2 * np.pi * (x + y)), np.ones_like(x), np.ones_like(x), np.ones_like(x)


def exact_smooth_density(x, y, t):
    return 1.0 + 0.2 * np.sin(2 * np.pi * (x + y - 2.0 * t))


def ic_paper_smooth(x, y):
    rho = 1.0 - 0.9999 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    return rho, np.ones_like(x), np.zeros_like(x), np.ones_like(x)


def exact_paper_smooth_density(x, y, t):
    return 1.0 - 0.9999 * np.sin(2 * np.pi * (x - t)) * np.sin(2 * np.pi * y)


def ic_rarefy(x, y):
    u = np.where(x < 0.5, -2.0, 2.0)
    return np.ones_like(x), u, np.zeros_like(x), 0.4 * np.ones_like(x)


def ic_uniform(rho=1.3, u=0.3, v=-0.2, p=0.8):
    def f(x, y):
        one = np.ones_like(x)
        return rho * one, u * one, v * one, p * one
    return f


def ic_blast(n: int, half_width: float = 1.1, gamma: float = GAMMA, e_total: float = 0.979264):
    """Point-energy blast on an n x n grid of [-w,w]^2 (n even): the 4 cells
    touching the origin share e_total; elsewhere p = 1e-12."""
    h = 2.0 * half_width / n
    p_in = (gamma - 1.0) * (e_total / 4.0) / (h * h)

    def f(x, y):
        inside = (np.abs(x) < h) & (np.abs(y) < h)
        return np.ones_like(x), np.zeros_like(x), np.zeros_like(x), np.where(inside, p_in, 1e-12)
    return f


def ic_blast3d(n: int, half_width: float = 1.1, gamma: float = GAMMA, e_total: float = 0.979264):
    """The 3D point-energy blast on an n^3 grid of [-w,w]^3 (n even): the 8
    cells touching the origin share e_total; elsewhere p = 1e-12, rho = 1,
    at rest.  Returns f(x, y, z) -> (rho, u, v, w, p)."""
    h = 2.0 * half_width / n
    p_in = (gamma - 1.0) * (e_total / 8.0) / (h * h * h)

    def f(x, y, z):
        inside = (np.abs(x) < h) & (np.abs(y) < h) & (np.abs(z) < h)
        zero = np.zeros_like(x)
        return np.ones_like(x), zero, zero, zero, np.where(inside, p_in, 1e-12)
    return f


def tet_mesh(n: int, box=(0.0, 1.0, 0.0, 1.0, 0.0, 1.0), periodic: bool = False, jitter: float = 0.0,
             seed: int = 0, permute: bool = False):
    """Tetrahedra of an n^3 grid of boxes, each box cut into six along its
    main diagonal (Kuhn's subdivision: v0 = the low corner, then one unit
    step along each axis in the order of a permutation), so neighbouring
    boxes share their faces' triangles.  Returns (xyz[nv][3], tets[nt][4],
    vid[nv]): vertex positions, positively oriented tetrahedra (indices into
    xyz) and a vertex id that identifies periodic images (equal to the vertex
    index when periodic is False; with periodic=True the grid index is taken
    modulo n on every axis, so the two cells of a face across the period
    share its vertex ids).  jitter moves interior vertices by up to jitter
    times the spacing (U[-1,1] per coordinate, from the seed); periodic
    meshes are not jittered.  permute renumbers each cell's four vertices by
    one of the 12 even permutations (drawn from seed + 1), which keeps the
    orientation positive, so that neighbouring cells list a shared face's
    vertices in unrelated orders."""
    m = n + 1
    ax = [np.linspace(box[2 * d], box[2 * d + 1], m) for d in range(3)]
    I, J, K = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    idx = lambda i, j, k: (k * m + j) * m + i   # noqa: E731
    xyz = np.zeros((m ** 3, 3))
    xyz[idx(I, J, K).ravel(), 0] = ax[0][I.ravel()]
    xyz[idx(I, J, K).ravel(), 1] = ax[1][J.ravel()]
    xyz[idx(I, J, K).ravel(), 2] = ax[2][K.ravel()]
    if jitter > 0.0 and not periodic:
        h = np.array([(box[2 * d + 1] - box[2 * d]) / n for d in range(3)])
        r = uniform01(seed, 3 * m ** 3).reshape(m ** 3, 3) * 2.0 - 1.0
        inner = ((I > 0) & (I < n) & (J > 0) & (J < n) & (K > 0) & (K < n)).ravel()
        ii = idx(I, J, K).ravel()[inner]
        xyz[ii] += jitter * h * r[ii]
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    # boxes in (k, j, i) order with i fastest, six cells per box in the order of perms
    Kb, Jb, Ib = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = np.stack([Ib.ravel(), Jb.ravel(), Kb.ravel()], axis=1)
    tets = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for q, pm in enumerate(perms):
        c = base.copy()
        tets[:, q, 0] = idx(c[:, 0], c[:, 1], c[:, 2])
        for s_, a in enumerate(pm):
            c[:, a] += 1
            tets[:, q, s_ + 1] = idx(c[:, 0], c[:, 1], c[:, 2])
    tets = tets.reshape(-1, 4).astype(np.int32)
    p = xyz[tets]
    vol = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    neg = vol < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    if permute:
        even = np.array([p for p in __import__("itertools").permutations(range(4))
                         if sum(p[a] > p[b] for a in range(4) for b in range(a + 1, 4)) % 2 == 0])
        pick = (uniform01(seed + 1, len(tets)) * len(even)).astype(np.int64)
        tets = np.take_along_axis(tets, even[pick], axis=1).astype(np.int32)
    if periodic:
        vid = idx(I % n, J % n, K % n).ravel()
        vid_of = np.empty(m ** 3, dtype=np.int32)
        vid_of[idx(I, J, K).ravel()] = vid
    else:
        vid_of = np.arange(m ** 3, dtype=np.int32)
    return xyz, tets, vid_of


def ic_quadrants(seed: int):
    """Four-quadrant Riemann data on [0,1]^2 drawn from a per-problem seed:
    rho ~ U[0.1,2], p ~ U[0.01,2], u, v ~ U[-1,1] in each quadrant."""
    r = uniform01(seed, 16).reshape(4, 4)
    rho = 0.1 + 1.9 * r[:, 0]
    p = 0.01 + 1.99 * r[:, 1]
    u = -1.0 + 2.0 * r[:, 2]
    v = -1.0 + 2.0 * r[:, 3]

    def f(x, y):
        qd = (x >= 0.5).astype(np.int64) + 2 * (y >= 0.5).astype(np.int64)
        return rho[qd], u[qd], v[qd], p[qd]
    return f


def ensemble_sizes(count: int = 256, lo: int = 32, hi: int = 256, seed: int = 4242):
    """Per-problem grid sizes n_p ~ U{lo..hi} (n_p x n_p cells each)."""
    r = uniform01(seed, count)
    return (lo + np.floor(r * (hi - lo + 1))).astype(np.int64).clip(lo, hi)


def random_modal_state(N: int, ML: int, seed: int, amp: float = 0.3, gamma: float = GAMMA,
                       rho_range=(0.5, 2.0), p_range=(0.2, 2.0)):
    """Random modal coefficients Q[N][4][ML] with positive averages.

    Averages come from random primitive data (rho, u, v, p); every higher
    coefficient is U[-amp, amp] times the magnitude of its variable's
    average, so large amp drives point values negative and wakes the
    limiters."""
    r = uniform01(seed, N * (4 + 4 * ML)).reshape(N, 4 + 4 * ML)
    rho = rho_range[0] + (rho_range[1] - rho_range[0]) * r[:, 0]
    u = -1.0 + 2.0 * r[:, 1]
    v = -1.0 + 2.0 * r[:, 2]
    p = p_range[0] + (p_range[1] - p_range[0]) * r[:, 3]
    avg = np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)], axis=1)
    Q = np.zeros((N, 4, ML))
    Q[:, :, 0] = avg
    scale = np.abs(avg) + 0.1 * np.abs(avg[:, :1])
    hi = (2.0 * r[:, 4:].reshape(N, 4, ML) - 1.0) * amp
    Q[:, :, 1:] = hi[:, :, 1:] * scale[:, :, None]
    return Q


def random_modal_state3(N: int, ML: int, seed: int, amp: float = 0.3, gamma: float = GAMMA,
                        rho_range=(0.5, 2.0), p_range=(0.2, 2.0)):
    """Random modal coefficients Q[N][5][ML] of 3D cells, (rho, rho u, rho v,
    rho w, E), built like random_modal_state: random primitive averages, every
    higher coefficient U[-amp, amp] times its variable's average magnitude."""
    r = uniform01(seed, N * (5 + 5 * ML)).reshape(N, 5 + 5 * ML)
    rho = rho_range[0] + (rho_range[1] - rho_range[0]) * r[:, 0]
    u, v, w = (-1.0 + 2.0 * r[:, k] for k in (1, 2, 3))
    p = p_range[0] + (p_range[1] - p_range[0]) * r[:, 4]
    avg = np.stack([rho, rho * u, rho * v, rho * w, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)], axis=1)
    Q = np.zeros((N, 5, ML))
    Q[:, :, 0] = avg
    scale = np.abs(avg) + 0.1 * np.abs(avg[:, :1])
    hi = (2.0 * r[:, 5:].reshape(N, 5, ML) - 1.0) * amp
    Q[:, :, 1:] = hi[:, :, 1:] * scale[:, :, None]
    return Q


# ------------------------------------------------ shock diffraction over a step
def normal_shock_state(mach, rho0=1.4, p0=1.0, gamma=1.4):
    """Primitive state (rho, u, v, p) behind a normal shock of the given Mach
    number running in +x into gas at rest (rho0, p0): the Rankine-Hugoniot
    jump conditions."""
    m2 = mach * mach
    r = (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p = (2.0 * gamma * m2 - (gamma - 1.0)) / (gamma + 1.0)
    c0 = np.sqrt(gamma * p0 / rho0)
    return rho0 * r, mach * c0 * (1.0 - 1.0 / r), 0.0, p0 * p


DIFFRACTION_BOX = (0.0, 13.0, 0.0, 11.0)
DIFFRACTION_STEP = (1.0, 6.0)       # the step occupies [0, 1] x [0, 6]
DIFFRACTION_MACH = 5.09
# (left, right, bottom, top) codes: inflow on the left side (which the mesh
# keeps above the step only), transparent elsewhere; the step's faces are
# walls through the mask code
DIFFRACTION_BC = (3, 2, 2, 2)


def diffraction_mask(nx, ny):
    """mask[ny][nx] of the Cartesian cells kept on [0,13] x [0,11]: every cell
    whose centre is outside the step [0,1] x [0,6]."""
    x0, x1, y0, y1 = DIFFRACTION_BOX
    xc = x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx
    yc = y0 + (np.arange(ny) + 0.5) * (y1 - y0) / ny
    X, Y = np.meshgrid(xc, yc, indexing="xy")
    return ~((X < DIFFRACTION_STEP[0]) & (Y < DIFFRACTION_STEP[1]))


def ic_diffraction(x, y):
    """Gas at rest (rho 1.4, p 1) with the Mach 5.09 shock at x = 1 above the step."""
    r1, u1, _, p1 = normal_shock_state(DIFFRACTION_MACH)
    left = x < DIFFRACTION_STEP[0]
    return np.where(left, r1, 1.4), np.where(left, u1, 0.0), 0.0 * x, np.where(left, p1, 1.0)


# ------------------------------------------------ Sedov blast on a disk
SEDOV_RADIUS = 1.1
SEDOV_ENERGY = 0.979264


def disk_triangles(ntri: int, radius: float = SEDOV_RADIUS, jitter: float = 0.15, seed: int = 20160129):
    """Exactly ntri counter-clockwise triangles covering the polygon inscribed
    in the circle of the given radius: B points on the circle and the V points
    of a jittered triangular lattice closest to the centre, Delaunay
    triangulated (scipy).  All hull points lie on the circle, so Euler's
    formula fixes the count, ntri = 2 V + B - 2, and B and V are chosen for it.
    Returns xy [nv][2], tv [ntri][3] (boundary vertices first)."""
    from scipy.spatial import Delaunay

    def lattice(h):
        # rows y = j h sqrt(3)/2, odd rows shifted by h/2; the points inside r < radius - h/2
        mi = int(np.ceil(radius / h)) + 2
        mj = int(np.ceil(radius / (h * np.sqrt(3.0) / 2.0))) + 2
        jj, ii = np.meshgrid(np.arange(-mj, mj + 1), np.arange(-mi, mi + 1), indexing="ij")
        lat = np.stack([(ii + 0.5 * (jj & 1)) * h, jj * h * np.sqrt(3.0) / 2.0], axis=-1).reshape(-1, 2)
        return lat[np.hypot(lat[:, 0], lat[:, 1]) < radius - 0.5 * h]

    # the spacing at which the ring count that Euler's formula leaves, B = ntri + 2 - 2 V(h),
    # equals the natural one, 2 pi radius / h (bisection; V(h) falls as h grows)
    h0 = np.sqrt(np.pi * radius ** 2 * 4.0 / (np.sqrt(3.0) * ntri))
    lo, hi = 0.8 * h0, 1.25 * h0
    for _ in range(60):
        h = 0.5 * (lo + hi)
        if ntri + 2 - 2 * len(lattice(h)) < 2.0 * np.pi * radius / h:
            lo = h
        else:
            hi = h
    h = hi
    inner = lattice(h)
    B = ntri + 2 - 2 * len(inner)
    if B < 3:
        raise ValueError("disk_triangles: no admissible spacing")
    th = 2.0 * np.pi * np.arange(B) / B
    ring = radius * np.stack([np.cos(th), np.sin(th)], axis=1)
    rng = np.random.default_rng(seed)
    inner = inner + rng.uniform(-jitter, jitter, size=inner.shape) * h
    xy = np.concatenate([ring, inner])
    tv = Delaunay(xy).simplices.astype(np.int32)
    a, b, c = xy[tv[:, 0]], xy[tv[:, 1]], xy[tv[:, 2]]
    det = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    flip = det < 0
    tv[flip, 1], tv[flip, 2] = tv[flip, 2].copy(), tv[flip, 1].copy()
    if len(tv) != ntri:
        raise ValueError(f"disk_triangles: {len(tv)} triangles, expected {ntri}")
    # triangles in Z-curve order of their centroids (the triangulation's own
    # order is scattered; neighbours close in memory keep gathers local)
    cen = (xy[tv[:, 0]] + xy[tv[:, 1]] + xy[tv[:, 2]]) / 3.0
    ij = np.clip(((cen + radius) / (2.0 * radius) * 65535.0).astype(np.int64), 0, 65535)

    def spread(v):   # bits of a 16-bit integer to the even positions
        v = (v | (v << 8)) & 0x00FF00FF
        v = (v | (v << 4)) & 0x0F0F0F0F
        v = (v | (v << 2)) & 0x33333333
        return (v | (v << 1)) & 0x55555555

    order = np.argsort(spread(ij[:, 0]) | (spread(ij[:, 1]) << 1), kind="stable")
    return xy, np.ascontiguousarray(tv[order])


def ic_sedov_disk(ntri: int, radius: float = SEDOV_RADIUS, e_total: float = SEDOV_ENERGY, gamma: float = GAMMA):
    """Gas at rest, rho = 1, E = 1e-12, except E = e_total / (pi r_d^2) inside
    r_d = sqrt(pi radius^2 / ntri), the mesh's characteristic length."""
    r_d = np.sqrt(np.pi * radius ** 2 / ntri)
    e_in = e_total / (np.pi * r_d ** 2)

    def f(x, y):
        e = np.where(np.hypot(x, y) < r_d, e_in, 1e-12)
        z = 0.0 * x
        return 1.0 + z, z, z, (gamma - 1.0) * e
    return f
