"""Seeded synthetic workloads shaped like the paper's experiments.

Each workload fixes a mesh (lsinput.mesh), the wavenumber k, the contrast
m = 1 - n^2 at the quadrature nodes and on a Cartesian grid, the incident
plane-wave directions and the far-field angles.  Convention (Section 2 of the
paper writes Delta u + k^2 n u = 0 with m = 1 - n): the optical index n_opt of
a material enters squared, so a material of optical index n_opt has
m = 1 - n_opt^2 (n_opt = 1.5 gives the paper's benchmark contrast eta = 1.25).

No solver arithmetic lives here.
"""
from dataclasses import dataclass

import numpy as np

from .mesh import disk_mesh, inclusion_disk_mesh, open_resonator_mesh, star_mesh


@dataclass
class Workload:
    name: str
    mesh: object
    k: float
    m: np.ndarray            # [NQ] complex128 contrast at the nodes
    box: tuple               # (xmin, xmax, ymin, ymax) of the Cartesian grid
    nx: int
    ny: int
    m_grid: np.ndarray       # [ny * nx] complex128 contrast at grid nodes (row-major, x fastest)
    directions: np.ndarray   # [R] incident plane-wave angles
    ff_angles: np.ndarray    # [n_ff] far-field angles
    tol: float

    @property
    def grid_points(self):
        x0, x1, y0, y1 = self.box
        gx = x0 + (x1 - x0) * np.arange(self.nx) / (self.nx - 1)
        gy = y0 + (y1 - y0) * np.arange(self.ny) / (self.ny - 1)
        X, Y = np.meshgrid(gx, gy)
        return np.stack([X.ravel(), Y.ravel()], axis=1)


def _grid(box, nx, ny):
    x0, x1, y0, y1 = box
    gx = x0 + (x1 - x0) * np.arange(nx) / (nx - 1)
    gy = y0 + (y1 - y0) * np.arange(ny) / (ny - 1)
    X, Y = np.meshgrid(gx, gy)
    return X.ravel(), Y.ravel()


def constant_disk(k=5.0, n_opt=1.5, n_rings=6, nx=64, ny=64, box=(-1.2, 1.2, -1.2, 1.2),
                  directions=(0.0,), n_ff=64, tol=1e-10):
    """Unit disk of constant optical index n_opt (the paper's benchmark,
    Section 6.1); 6 n_rings^2 curved triangles (n_rings = 6: 216 triangles,
    3,240 nodes)."""
    mesh = disk_mesh(n_rings)
    mval = 1.0 - n_opt**2
    m = np.full(mesh.n_nodes, mval, dtype=np.complex128)
    X, Y = _grid(box, nx, ny)
    m_grid = np.where(X**2 + Y**2 < 1.0, mval, 0.0).astype(np.complex128)
    return Workload("disk", mesh, float(k), m, box, nx, ny, m_grid,
                    np.asarray(directions, float), 2 * np.pi * np.arange(n_ff) / n_ff, tol)


def _two_material_index(x, y, inside_incl):
    n_bg = 1.5 + 0.2 * np.exp(-(x**2 + y**2) / 0.1)
    return np.where(inside_incl, 2.2, n_bg)


def two_material(level="small", k=20.0, nx=256, ny=256, box=(-1.2, 1.2, -1.2, 1.2),
                 directions=(np.pi / 4,), n_ff=64, tol=1e-8):
    """Unit disk with an off-centre circular inclusion (radius 0.3 at (0.3, 0.1));
    n_opt = 1.5 + 0.2 exp(-|x|^2 / 0.1) outside the inclusion and 2.2 inside
    (a jump across the interface).  Levels: 'tiny' 120 triangles, 'small'
    2,680 triangles (40,200 nodes), 'medium' 13,042 (195,630), 'large'
    32,830 (492,450)."""
    sizes = {"tiny": (2, 3, 16), "small": (6, 14, 88), "medium": (13, 31, 194),
             "large": (21, 49, 308)}
    nr, ns, nth = sizes[level]
    mesh = inclusion_disk_mesh(nr, ns, nth)
    x, y = mesh.nodes[:, 0], mesh.nodes[:, 1]
    inside = mesh.node_domain == 1
    m = (1.0 - _two_material_index(x, y, inside) ** 2).astype(np.complex128)
    X, Y = _grid(box, nx, ny)
    in_disk = X**2 + Y**2 < 1.0
    in_incl = (X - 0.3) ** 2 + (Y - 0.1) ** 2 < 0.09
    m_grid = np.where(in_disk, 1.0 - _two_material_index(X, Y, in_incl) ** 2, 0.0).astype(np.complex128)
    return Workload("two_material_" + level, mesh, float(k), m, box, nx, ny, m_grid,
                    np.asarray(directions, float), 2 * np.pi * np.arange(n_ff) / n_ff, tol)


def perturbed_contrast(wl, amp=0.05, center=(-0.3, -0.2), width=0.02):
    """Contrast of the differentiation form's target medium: the two-material index
    plus a Gaussian blob amp exp(-|x - center|^2 / width) (m = 1 - n_opt^2)."""
    x, y = wl.mesh.nodes[:, 0], wl.mesh.nodes[:, 1]
    n_opt = np.sqrt(1.0 - wl.m.real)
    n_opt = n_opt + amp * np.exp(-((x - center[0]) ** 2 + (y - center[1]) ** 2) / width)
    return (1.0 - n_opt**2).astype(np.complex128)


def star_scatterer(s, n_nodes_target, k=None, nx=128, ny=128, n_dirs=64, n_ff=64, tol=1e-8):
    """Scatterer s of the batched workload: star r = 1 + 0.2 cos(5 theta + phi_s)
    with phi_s ~ U[0, 2 pi) from default_rng(20261202 + s), an inner interface at
    half the radius, n_opt = 1.3 + 0.3 exp(-|x - c_s|^2 / 0.1) plus 0.5 inside
    the interface, c_s = 0.2 (cos phi_s, sin phi_s); k given, else (10, 20, 40)[s % 3]
    (the batching configuration passes k by scatterer size)."""
    rng = np.random.default_rng(20261202 + s)
    phi = float(rng.uniform(0.0, 2 * np.pi))
    if k is None:
        k = (10.0, 20.0, 40.0)[s % 3]
    n_tri = max(n_nodes_target // 15, 24)
    # split: inner core (6 nr^2) gets ~1/4 of the triangles, shell the rest
    nr = max(1, int(round(np.sqrt(n_tri / 4 / 6))))
    shell = n_tri - 6 * nr * nr
    nth = max(12, int(round(np.sqrt(shell * 2 * np.pi / 0.5 / 2))))
    ns = max(1, int(round(shell / (2 * nth))))
    mesh = star_mesh(phi, nr, ns, nth)
    c = 0.2 * np.array([np.cos(phi), np.sin(phi)])
    x, y = mesh.nodes[:, 0], mesh.nodes[:, 1]
    n_opt = 1.3 + 0.3 * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2) / 0.1) + 0.5 * (mesh.node_domain == 1)
    m = (1.0 - n_opt**2).astype(np.complex128)
    box = (-1.45, 1.45, -1.45, 1.45)
    X, Y = _grid(box, nx, ny)
    th = np.arctan2(Y, X)
    r = np.hypot(X, Y)
    rb = 1.0 + 0.2 * np.cos(5 * th + phi)
    ng = 1.3 + 0.3 * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2) / 0.1) + 0.5 * (r < 0.5 * rb)
    m_grid = np.where(r < rb, 1.0 - ng**2, 0.0).astype(np.complex128)
    dirs = 2 * np.pi * np.arange(n_dirs) / n_dirs
    return Workload(f"star{s}", mesh, float(k), m, box, nx, ny, m_grid, dirs,
                    2 * np.pi * np.arange(n_ff) / n_ff, tol)


def open_resonator(k=10.0, n_s=3, n_theta=60, nx=96, ny=96, box=(-1.2, 1.2, -1.2, 1.2), n_ff=64, tol=1e-10):
    """The paper's open-cavity resonator (Section 6, more general examples): the truncated
    annulus 0.8 < |x| < 1, |theta| > 20 degrees, with the radial contrast
    m(x) = exp(-((|x| - 0.9) / 0.1201)^2) inside (m given directly), a plane wave along
    d = (-1, 0) entering the cavity through its aperture; k kept small here (the paper
    runs k = 200)."""
    th0 = np.pi / 9
    mesh = open_resonator_mesh(n_s, n_theta, theta0=th0)
    r = np.hypot(mesh.nodes[:, 0], mesh.nodes[:, 1])
    m = np.exp(-(((r - 0.9) / 0.1201) ** 2)).astype(np.complex128)
    X, Y = _grid(box, nx, ny)
    R = np.hypot(X, Y)
    inside = (R > 0.8) & (R < 1.0) & (np.abs(np.arctan2(Y, X)) > th0)
    m_grid = np.where(inside, np.exp(-(((R - 0.9) / 0.1201) ** 2)), 0.0).astype(np.complex128)
    return Workload("open_resonator", mesh, float(k), m, box, nx, ny, m_grid, np.array([np.pi]),
                    2 * np.pi * np.arange(n_ff) / n_ff, tol)


def random_density(n, seed):
    """Seeded complex test vector with entries of modulus <= 1."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)).astype(np.complex128)
