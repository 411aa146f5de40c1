"""Seeded synthetic inputs: triangle meshes and initial states.

This module is shared by the CUDA path's tests and benchmark and by the
oracle's tests.  It holds none of the method's arithmetic: it only draws
meshes (jittered lattices split on random diagonals) and evaluates the
initial conditions of the paper's test problems (isentropic vortex,
Section 3.1; 2D Riemann problem; 2D Sod problem, Section 3.2).

Every generator takes an explicit seed and uses numpy's PCG64
(``numpy.random.default_rng``), so both sides of a parity test see the
same bytes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = 1.4


@dataclass
class Mesh:
    """A triangle mesh as plain arrays (original vertex ids)."""

    xy: np.ndarray  # [nv, 2] float64
    tri: np.ndarray | tuple  # [nt, 3] int32 counter-clockwise, or (cell_off, cell_vtx) of a hybrid mesh
    Lx: float  # periodic length in x (0 = not periodic)
    Ly: float  # periodic length in y (0 = not periodic)
    n: int = 0  # lattice size it was drawn from (informational)
    h: float = 0.0  # lattice spacing (informational)
    ghost_donor: np.ndarray | None = None  # [nv] donor of each ghost vertex, -1 for real ones

    @property
    def nv(self) -> int:
        return int(self.xy.shape[0])

    @property
    def nt(self) -> int:
        if isinstance(self.tri, tuple):
            return int(self.tri[0].shape[0] - 1)
        return int(self.tri.shape[0])


def _signed_areas(xy, tri, Lx, Ly):
    a = xy[tri[:, 0]]
    b = xy[tri[:, 1]] - a
    c = xy[tri[:, 2]] - a
    if Lx > 0:
        b[:, 0] -= Lx * np.rint(b[:, 0] / Lx)
        c[:, 0] -= Lx * np.rint(c[:, 0] / Lx)
    if Ly > 0:
        b[:, 1] -= Ly * np.rint(b[:, 1] / Ly)
        c[:, 1] -= Ly * np.rint(c[:, 1] / Ly)
    return 0.5 * (b[:, 0] * c[:, 1] - b[:, 1] * c[:, 0])


def torus_lattice(n: int, L: float = 10.0, jitter: float = 0.2, seed: int = 1001,
                  random_diagonals: bool = True, origin: float = 0.0) -> Mesh:
    """n x n vertices on the periodic square [origin, origin+L)^2.

    Vertex (i, j) has id j*n + i and sits at (origin + i*h, origin + j*h),
    h = L/n, moved by U(-jitter*h, +jitter*h) in x and y independently.
    Each lattice quad is split on a Bernoulli(1/2) diagonal (or always on
    the (i,j)-(i+1,j+1) diagonal when ``random_diagonals`` is False).
    """
    if n < 4:
        raise ValueError("torus lattice needs n >= 4")
    rng = np.random.default_rng(seed)
    h = L / n
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    xy = np.stack([origin + ii.ravel() * h, origin + jj.ravel() * h], axis=1).astype(np.float64)
    if jitter > 0:
        xy += rng.uniform(-jitter * h, jitter * h, size=xy.shape)
    diag = rng.integers(0, 2, size=n * n) if random_diagonals else np.zeros(n * n, np.int64)
    i = ii.ravel()
    j = jj.ravel()
    a = j * n + i
    b = j * n + (i + 1) % n
    c = ((j + 1) % n) * n + (i + 1) % n
    d = ((j + 1) % n) * n + i
    t0 = np.where(diag[:, None] == 0, np.stack([a, b, c], 1), np.stack([a, b, d], 1))
    t1 = np.where(diag[:, None] == 0, np.stack([a, c, d], 1), np.stack([b, c, d], 1))
    tri = np.concatenate([t0, t1], 0).astype(np.int32)
    m = Mesh(xy=xy, tri=tri, Lx=L, Ly=L, n=n, h=h)
    if np.any(_signed_areas(xy, tri, L, L) <= 0):
        raise ValueError("jittered lattice produced a non-positive triangle")
    return m


def hybrid_lattice(n: int, L: float = 10.0, jitter: float = 0.2, seed: int = 1007, tri_fraction: float = 0.5,
                   origin: float = 0.0) -> Mesh:
    """Hybrid triangle / quadrilateral mesh on the periodic square.

    The n x n torus lattice of ``torus_lattice`` (same ids, spacing and
    jitter); each lattice quad is kept as a counter-clockwise
    quadrilateral (a, b, c, d) or, with probability ``tri_fraction``, split
    on a Bernoulli(1/2) diagonal into two triangles.  ``tri`` is returned as
    the CSR pair (cell_off int64 [nc+1], cell_vtx int32).
    """
    if n < 4:
        raise ValueError("torus lattice needs n >= 4")
    rng = np.random.default_rng(seed)
    h = L / n
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    xy = np.stack([origin + ii.ravel() * h, origin + jj.ravel() * h], axis=1).astype(np.float64)
    if jitter > 0:
        xy += rng.uniform(-jitter * h, jitter * h, size=xy.shape)
    split = rng.uniform(size=n * n) < tri_fraction
    diag = rng.integers(0, 2, size=n * n)
    i, j = ii.ravel(), jj.ravel()
    a = j * n + i
    b = j * n + (i + 1) % n
    c = ((j + 1) % n) * n + (i + 1) % n
    d = ((j + 1) % n) * n + i
    off, vtx = [0], []
    for q in range(n * n):
        if not split[q]:
            vtx += [a[q], b[q], c[q], d[q]]
            off.append(off[-1] + 4)
        elif diag[q] == 0:
            vtx += [a[q], b[q], c[q], a[q], c[q], d[q]]
            off += [off[-1] + 3, off[-1] + 6]
        else:
            vtx += [a[q], b[q], d[q], b[q], c[q], d[q]]
            off += [off[-1] + 3, off[-1] + 6]
    return Mesh(xy=xy, tri=(np.array(off, np.int64), np.array(vtx, np.int32)), Lx=L, Ly=L, n=n, h=h)


def union_jack_lattice(n: int, L: float = 10.0) -> Mesh:
    """The n x n torus lattice (n even) with each quad split on the diagonal
    through its corner (i, j) when i + j is even and through (i+1, j)
    otherwise: vertices with i + j even have 8 neighbours, the others 4
    (the valence-4 configuration of Fig. l1-tria4)."""
    if n < 4 or n % 2:
        raise ValueError("union jack lattice needs an even n >= 4")
    h = L / n
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    xy = np.stack([ii.ravel() * h, jj.ravel() * h], axis=1).astype(np.float64)
    i, j = ii.ravel(), jj.ravel()
    a = j * n + i
    b = j * n + (i + 1) % n
    c = ((j + 1) % n) * n + (i + 1) % n
    d = ((j + 1) % n) * n + i
    even = ((i + j) % 2 == 0)[:, None]
    t0 = np.where(even, np.stack([a, b, c], 1), np.stack([a, b, d], 1))
    t1 = np.where(even, np.stack([a, c, d], 1), np.stack([b, c, d], 1))
    tri = np.concatenate([t0, t1], 0).astype(np.int32)
    return Mesh(xy=xy, tri=tri, Lx=L, Ly=L, n=n, h=h)


def box_lattice(n: int, ghost_layers: int = 0, jitter: float = 0.2, seed: int = 1003,
                random_diagonals: bool = True) -> Mesh:
    """Lattice on [0,1]^2 with n points per side (spacing h = 1/(n-1)).

    ``ghost_layers`` extra lattice layers are added outside the unit
    square on every side.  Only vertices strictly inside the square are
    jittered; vertices on the square's boundary and in the ghost layers
    stay on the lattice.  Quads are split on Bernoulli(1/2) diagonals.
    Vertex (i, j), i, j in [-g, n-1+g], has id (j+g)*m + (i+g), m = n+2g.
    """
    g = ghost_layers
    h = 1.0 / (n - 1)
    m = n + 2 * g
    rng = np.random.default_rng(seed)
    jj, ii = np.meshgrid(np.arange(-g, n + g), np.arange(-g, n + g), indexing="ij")
    i = ii.ravel()
    j = jj.ravel()
    xy = np.stack([i * h, j * h], axis=1).astype(np.float64)
    jit = rng.uniform(-jitter * h, jitter * h, size=xy.shape)
    interior = (i > 0) & (i < n - 1) & (j > 0) & (j < n - 1)
    xy[interior] += jit[interior]
    diag = rng.integers(0, 2, size=(m - 1) * (m - 1))
    if not random_diagonals:
        diag[:] = 0
    qi, qj = np.meshgrid(np.arange(m - 1), np.arange(m - 1), indexing="xy")
    qi = qi.ravel()
    qj = qj.ravel()
    a = qj * m + qi
    b = qj * m + qi + 1
    c = (qj + 1) * m + qi + 1
    d = (qj + 1) * m + qi
    t0 = np.where(diag[:, None] == 0, np.stack([a, b, c], 1), np.stack([a, b, d], 1))
    t1 = np.where(diag[:, None] == 0, np.stack([a, c, d], 1), np.stack([b, c, d], 1))
    tri = np.concatenate([t0, t1], 0).astype(np.int32)
    mesh = Mesh(xy=xy, tri=tri, Lx=0.0, Ly=0.0, n=n, h=h)
    if np.any(_signed_areas(xy, tri, 0.0, 0.0) <= 0):
        raise ValueError("jittered box lattice produced a non-positive triangle")
    # ghost vertex -> the boundary lattice vertex nearest to it (-1 for real vertices)
    ci = np.clip(i, 0, n - 1)
    cj = np.clip(j, 0, n - 1)
    donor = ((cj + g) * m + (ci + g)).astype(np.int32)
    donor[interior | ((i >= 0) & (i <= n - 1) & (j >= 0) & (j <= n - 1))] = -1
    mesh.ghost_donor = donor
    return mesh


def channel_lattice(n: int, x0: float = -65.0, x1: float = 15.0, Ly: float = 80.0, ghost_layers: int = 5,
                    jitter: float = 0.0, seed: int = 1009, random_diagonals: bool = False) -> Mesh:
    """Lattice on [x0, x1] x [0, Ly) periodic in y, with Dirichlet ghost
    layers outside x0 and x1.

    Spacing h = Ly / n in both directions (x1 - x0 must be a multiple of
    h); ``ghost_layers`` lattice columns are added beyond each x boundary.
    Vertex (i, j), i in [-g, nx-1+g] with nx = (x1-x0)/h + 1, j in [0, n),
    has id j*m + (i+g), m = nx + 2g, at (x0 + i h, j h - Ly/2) (so y spans
    [-Ly/2, Ly/2)).  Only vertices strictly inside (x0, x1) are jittered.
    Each ghost is its own donor (``ghost_donor[v] = v``): a Dirichlet vertex
    that keeps the state it is given.
    """
    h = Ly / n
    nx = int(round((x1 - x0) / h)) + 1
    if abs((nx - 1) * h - (x1 - x0)) > 1e-9 * (x1 - x0):
        raise ValueError("x1 - x0 must be a multiple of Ly / n")
    g = ghost_layers
    m = nx + 2 * g
    rng = np.random.default_rng(seed)
    jj, ii = np.meshgrid(np.arange(n), np.arange(-g, nx + g), indexing="ij")
    i, j = ii.ravel(), jj.ravel()
    xy = np.stack([x0 + i * h, j * h - 0.5 * Ly], axis=1).astype(np.float64)
    inside = (i > 0) & (i < nx - 1)
    if jitter > 0:
        xy[inside] += rng.uniform(-jitter * h, jitter * h, size=(int(inside.sum()), 2))
    qi, qj = np.meshgrid(np.arange(m - 1), np.arange(n), indexing="xy")
    qi, qj = qi.ravel(), qj.ravel()
    a = qj * m + qi
    b = qj * m + qi + 1
    c = ((qj + 1) % n) * m + qi + 1
    d = ((qj + 1) % n) * m + qi
    diag = rng.integers(0, 2, size=a.size) if random_diagonals else np.zeros(a.size, np.int64)
    t0 = np.where(diag[:, None] == 0, np.stack([a, b, c], 1), np.stack([a, b, d], 1))
    t1 = np.where(diag[:, None] == 0, np.stack([a, c, d], 1), np.stack([b, c, d], 1))
    tri = np.concatenate([t0, t1], 0).astype(np.int32)
    mesh = Mesh(xy=xy, tri=tri, Lx=0.0, Ly=Ly, n=n, h=h)
    if np.any(_signed_areas(xy, tri, 0.0, Ly) <= 0):
        raise ValueError("channel lattice produced a non-positive triangle")
    ids = np.arange(xy.shape[0], dtype=np.int32)
    mesh.ghost_donor = np.where((i < 0) | (i > nx - 1), ids, -1).astype(np.int32)
    return mesh


def shock_vortex(xy, gamma=GAMMA, mach_shock=1.2, mach_vortex=1.0, centre=(4.0, 0.0), Ly=80.0):
    """Shock-vortex interaction of Section 3.2: a stationary normal shock at
    x = 0 with the supersonic state (rho, u, v, p) = (1, -M_s, 0, 1/gamma)
    (sound speed 1) on x >= 0 and the Rankine-Hugoniot state on x < 0, and
    the isentropic vortex of the paper's formula centred at ``centre`` on
    the upstream side: rho = (1 - (gamma-1)/2 M_v^2 e^(1-r^2))^(1/(gamma-1)),
    p = rho^gamma / gamma, (du, dv) = M_v e^((1-r^2)/2) (-y', x')."""
    M = mach_shock
    r2r1 = (gamma + 1) * M * M / ((gamma - 1) * M * M + 2)
    p2p1 = 1 + 2 * gamma / (gamma + 1) * (M * M - 1)
    x, y = xy[:, 0], xy[:, 1]
    pre = x >= 0
    rho = np.where(pre, 1.0, r2r1)
    u = np.where(pre, -M, -M / r2r1)
    v = np.zeros_like(x)
    p = np.where(pre, 1.0 / gamma, p2p1 / gamma)
    dx = x - centre[0]
    dy = y - centre[1]
    if Ly > 0:
        dy -= Ly * np.rint(dy / Ly)
    r2 = dx * dx + dy * dy
    rv = (1 - 0.5 * (gamma - 1) * mach_vortex ** 2 * np.exp(1 - r2)) ** (1 / (gamma - 1))
    amp = mach_vortex * np.exp(0.5 * (1 - r2))
    rho = np.where(pre, rv, rho)
    p = np.where(pre, rv ** gamma / gamma, p)
    u = np.where(pre, u - amp * dy, u)
    v = np.where(pre, amp * dx, v)
    return primitive_to_conservative(rho, u, v, p, gamma)


def shock_vortex_case(n: int = 160, ghost_layers: int = 5, jitter: float = 0.0, random_diagonals: bool = False):
    """The shock-vortex problem on [-65, 15] x [-40, 40] (n points across the
    periodic y period; the paper's finest spacing 0.08 is n = 1000)."""
    mesh = channel_lattice(n, -65.0, 15.0, 80.0, ghost_layers, jitter=jitter, random_diagonals=random_diagonals)
    return mesh, shock_vortex(mesh.xy)


def permute_vertices(mesh: Mesh, seed: int) -> tuple[Mesh, np.ndarray]:
    """Return the same mesh with vertex ids shuffled, and the permutation.

    ``perm[new_id] = old_id``.
    """
    rng = np.random.default_rng(seed)
    perm = rng.permutation(mesh.nv)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(mesh.nv)
    tri = inv[mesh.tri].astype(np.int32)
    return Mesh(xy=mesh.xy[perm].copy(), tri=tri, Lx=mesh.Lx, Ly=mesh.Ly, n=mesh.n, h=mesh.h), perm


# --------------------------------------------------------------------------
# Initial conditions (primitive -> conservative records [nv][4] = rho, rho*u,
# rho*v, rho*E with E = e + (u^2+v^2)/2 and p = (gamma-1) rho e, Section 2.1)
# --------------------------------------------------------------------------

def primitive_to_conservative(rho, u, v, p, gamma=GAMMA):
    w = np.empty((np.size(rho), 4), np.float64)
    w[:, 0] = rho
    w[:, 1] = rho * u
    w[:, 2] = rho * v
    w[:, 3] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return w


def _min_image(d, L):
    if L > 0:
        return d - L * np.rint(d / L)
    return d


def isentropic_vortex(xy, L=10.0, beta=5.0, centre=(5.0, 5.0), t=0.0, gamma=GAMMA,
                      u_inf=1.0, v_inf=1.0):
    """Isentropic vortex of Section 3.1 (free stream rho=u=v=p=1).

    At time t the exact solution is the initial vortex translated by
    (u_inf*t, v_inf*t), wrapped into the periodic box of side L.
    Distances use the minimum image.
    """
    xc = centre[0] + u_inf * t
    yc = centre[1] + v_inf * t
    xb = _min_image(xy[:, 0] - xc, L)
    yb = _min_image(xy[:, 1] - yc, L)
    r2 = xb * xb + yb * yb
    rho = (1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)) ** (1.0 / (gamma - 1.0))
    amp = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u = u_inf - amp * yb
    v = v_inf + amp * xb
    p = rho ** gamma
    return primitive_to_conservative(rho, u, v, p, gamma)


RIEMANN_2D_QUADRANTS = (
    # (rho, u, v, p) for x>1/2,y>1/2 ; x<1/2,y>1/2 ; x<1/2,y<1/2 ; x>1/2,y<1/2
    (1.5, 0.0, 0.0, 1.5),
    (0.5323, 1.206, 0.0, 0.3),
    (0.138, 1.206, 1.206, 0.029),
    (0.5323, 0.0, 1.206, 0.3),
)


def riemann_2d(xy, gamma=GAMMA):
    """Four-quadrant 2D Riemann problem on [0,1]^2, interface at x=y=1/2."""
    x = xy[:, 0]
    y = xy[:, 1]
    q = np.where(x > 0.5, np.where(y > 0.5, 0, 3), np.where(y > 0.5, 1, 2))
    tab = np.array(RIEMANN_2D_QUADRANTS)
    s = tab[q]
    return primitive_to_conservative(s[:, 0], s[:, 1], s[:, 2], s[:, 3], gamma)


def sod_2d(xy, gamma=GAMMA):
    """2D Sod problem of Section 3.2 on [-1,1]^2: (1,0,0,1) inside |x|,|y|<1/4."""
    inside = (np.abs(xy[:, 0]) < 0.25) & (np.abs(xy[:, 1]) < 0.25)
    rho = np.where(inside, 1.0, 0.125)
    p = np.where(inside, 1.0, 0.1)
    z = np.zeros_like(rho)
    return primitive_to_conservative(rho, z, z, p, gamma)


def vortex_case(n: int, seed: int = 1001, L: float = 10.0, beta: float = 5.0,
                centre=(5.0, 5.0), jitter: float = 0.2, random_diagonals: bool = True):
    """Periodic vortex workload: jittered torus lattice + vortex state."""
    mesh = torus_lattice(n, L=L, jitter=jitter, seed=seed, random_diagonals=random_diagonals)
    w0 = isentropic_vortex(mesh.xy, L=L, beta=beta, centre=centre)
    return mesh, w0


def riemann_case(n: int, ghost_layers: int = 5, seed: int = 1003, jitter: float = 0.2,
                 random_diagonals: bool = True):
    """Four-quadrant Riemann problem on [0,1]^2 with transmissive ghost layers."""
    mesh = box_lattice(n, ghost_layers=ghost_layers, seed=seed, jitter=jitter, random_diagonals=random_diagonals)
    w0 = riemann_2d(mesh.xy)
    return mesh, w0


def sod_case(n: int = 55, jitter: float = 0.0, random_diagonals: bool = False, seed: int = 1006):
    """2D Sod problem of Section 3.2 on the periodic square [-1,1]^2 (n x n
    lattice; 55 x 55 = 3025 points against the paper's 3058)."""
    mesh = torus_lattice(n, L=2.0, jitter=jitter, seed=seed, random_diagonals=random_diagonals, origin=-1.0)
    return mesh, sod_2d(mesh.xy)


def batch_sizes(count: int = 64, lo: float = 5e3, hi: float = 2e5, seed: int = 2004):
    """Log-uniform mesh sizes, vortex strengths in [1,5], centres in [3,7]^2."""
    rng = np.random.default_rng(seed)
    v = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count)))
    n = np.maximum(8, np.rint(np.sqrt(v))).astype(int)
    beta = rng.uniform(1.0, 5.0, size=count)
    centres = rng.uniform(3.0, 7.0, size=(count, 2))
    return n, beta, centres


def random_state_perturbation(nv: int, scale: float, seed: int):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((nv, 4))
