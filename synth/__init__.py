"""Seeded synthetic microstructures and workloads for the FFT phase-field-fracture RVE.

This module is shared by the oracle, the tests and the benchmark. It only *describes* inputs:
voxel phase maps, per-grain lattice constants, orientations, local toughness, cleavage normals and
the initial crack. It holds none of the method's arithmetic: no stiffness rotation, no FFT, no
energy, no solver. Each consumer (the FP64 oracle and the CUDA library) turns the description
into its own tables.

Conventions
-----------
* Grid ``n = (nx, ny, nz)``; 2D problems have ``nz == 1`` and ``dim == 2``. Voxel size h = 1, so
  lengths (``ell``, radii, crack lengths) are in voxels.
* ``grain_id`` is int32 with numpy shape ``(nz, ny, nx)``: x varies fastest in memory.
* Lattice stiffness of grain g is cubic, given by the tensor constants
  ``C_cubic[g] = (C1111, C1122, C1212)``. An isotropic phase with Young modulus E and Poisson
  ratio nu has C1111 = lam + 2 mu, C1122 = lam, C1212 = mu (3D Lame constants; 2D problems are
  plane strain).
* ``R[g]`` rotates lattice axes to sample axes (the tensor R of Eq. (Crot), Sec. 2.2).
* ``cleave_n[g]`` is the weak-plane normal in lattice axes and ``beta[g]`` the cleavage weight of
  Eq. (PFFani); beta = 0 means isotropic damage.
* The initial crack is a row of voxels at ``y = crack.row`` spanning ``x0 .. x0+length-1``
  (all z in 3D), the "row of voxels with negligible stiffness" of Sec. 4.3.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Crack", "Microstructure", "Workload", "iso_constants", "homogeneous", "laminate", "fibres",
    "voronoi", "inplane_rotations", "so3_rotations", "homogeneous_plate_64", "fibre_composite_512",
    "polycrystal_1024", "batched_3d_polycrystals", "serving_stream", "small_cases",
]

CRACK_NONE, CRACK_CTE, CRACK_CPFE = 0, 1, 2


@dataclass
class Crack:
    """Initial crack: a voxel row of reduced stiffness plus its initial damage recipe (Sec. 4.3).

    kind: CRACK_NONE (no notch, no enrichment), CRACK_CTE (phi_disc = 1 at the two tip voxels,
    Eq. (damini)) or CRACK_CPFE (phi_disc = 1 on every crack voxel).
    """
    kind: int = CRACK_NONE
    row: int = 0
    x0: int = 0
    length: int = 0
    phi_M: float = 0.8
    stiffness: float = 1e-6

    def mask(self, n):
        nx, ny, nz = n
        m = np.zeros((nz, ny, nx), dtype=bool)
        if self.kind != CRACK_NONE and self.length > 0:
            xs = (self.x0 + np.arange(self.length)) % nx
            m[:, self.row, xs] = True
        return m


@dataclass
class Microstructure:
    n: tuple
    dim: int
    grain_id: np.ndarray
    C_cubic: np.ndarray
    R: np.ndarray
    Gc: np.ndarray
    cleave_n: np.ndarray
    beta: np.ndarray
    crack: Crack = field(default_factory=Crack)
    name: str = ""

    @property
    def n_grains(self):
        return int(self.C_cubic.shape[0])

    @property
    def nvox(self):
        return int(self.n[0] * self.n[1] * self.n[2])

    def validate(self):
        nx, ny, nz = self.n
        assert self.grain_id.shape == (nz, ny, nx) and self.grain_id.dtype == np.int32
        g = self.n_grains
        assert self.C_cubic.shape == (g, 3) and self.R.shape == (g, 3, 3)
        assert self.Gc.shape == (g,) and self.cleave_n.shape == (g, 3) and self.beta.shape == (g,)
        assert self.grain_id.min() >= 0 and self.grain_id.max() < g
        assert self.dim in (2, 3) and (self.dim == 3 or nz == 1)
        return self


@dataclass
class Workload:
    """A microstructure plus the solver parameters one toughness run uses."""
    micro: Microstructure
    ell: float
    k_res: float = 1e-6
    split: int = 0           # 0: no split (the paper's model); 1: spectral split (isotropic only)
    n_inc: int = 100
    dtau: float = 0.0
    f: tuple = (0.0, 1.0, 0.0, 0.0, 0.0, 0.0)   # xx, yy, zz, yz, xz, xy tensor components
    precision: str = "fp64"
    name: str = ""

    @property
    def A_g(self):
        """Reference crack length (2D) or area (3D) of Eq. (JaviGc0): the new crack only."""
        m = self.micro
        nx, ny, nz = m.n
        a0 = m.crack.length if m.crack.kind != CRACK_NONE else 0
        return float((nx - a0) * (nz if m.dim == 3 else 1))


def iso_constants(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return (lam + 2.0 * mu, lam, mu)


def _micro(n, dim, gid, C, R=None, Gc=None, cleave=None, beta=None, crack=None, name=""):
    g = len(C)
    C = np.asarray(C, dtype=np.float64).reshape(g, 3)
    R = np.repeat(np.eye(3)[None], g, 0) if R is None else np.asarray(R, np.float64).reshape(g, 3, 3)
    Gc = np.ones(g) if Gc is None else np.asarray(Gc, np.float64).reshape(g)
    cleave = np.tile([1.0, 0.0, 0.0], (g, 1)) if cleave is None else np.asarray(cleave, np.float64).reshape(g, 3)
    beta = np.zeros(g) if beta is None else np.asarray(beta, np.float64).reshape(g)
    return Microstructure(tuple(int(v) for v in n), dim, np.ascontiguousarray(gid, dtype=np.int32),
                          C, R, Gc, cleave, beta, crack or Crack(), name).validate()


def _grid(n):
    n = tuple(int(v) for v in n)
    if len(n) == 2:
        return (n[0], n[1], 1), 2
    return n, 3


def homogeneous(n, E=1.0, nu=0.3, Gc=1.0, crack=None, name="homogeneous"):
    n3, dim = _grid(n)
    gid = np.zeros(n3[::-1], np.int32)
    return _micro(n3, dim, gid, [iso_constants(E, nu)], Gc=[Gc], crack=crack, name=name)


def laminate(n, axis, widths, phases, crack=None, name="laminate"):
    """Layers stacked along ``axis`` ('x' or 'y'); ``widths`` voxels each, repeating.

    ``phases`` is a list of (E, nu, Gc), one per layer in ``widths``.
    """
    n3, dim = _grid(n)
    nx, ny, nz = n3
    ax_len = nx if axis == "x" else ny
    assert sum(widths) == ax_len
    layer = np.repeat(np.arange(len(widths)), widths)
    gid = np.zeros((nz, ny, nx), np.int32)
    if axis == "x":
        gid[:] = layer[None, None, :]
    else:
        gid[:] = layer[None, :, None]
    C = [iso_constants(E, nu) for (E, nu, _) in phases]
    Gc = [gc for (_, _, gc) in phases]
    return _micro(n3, dim, gid, C, Gc=Gc, crack=crack, name=name)


def _periodic_dist2(pts, centre, n):
    d = np.abs(pts - centre)
    d = np.minimum(d, np.asarray(n, np.float64) - d)
    return (d * d).sum(-1)


def fibres(n, radius, vf, seed, E_m=1.0, E_f=5.0, nu=0.3, Gc_m=1.0, Gc_f=2.0, crack=None,
           crack_clearance=0.0, gap=1.0, max_tries=200000, name="fibres"):
    """Random sequential addition of non-overlapping periodic discs (2D).

    Discs of radius ``radius`` are placed uniformly at random (seeded), rejected when closer than
    2 r + gap to an accepted disc (periodic minimum image) or when their centre lies within
    r + ``crack_clearance`` of the crack segment, until the voxel fraction reaches ``vf``. A voxel
    whose centre lies at distance <= r from a disc centre is fibre (grain 1); the matrix is grain 0.
    """
    n3, dim = _grid(n)
    nx, ny, _ = n3
    assert dim == 2
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    pts = np.stack([xx, yy], -1)
    fib = np.zeros((ny, nx), bool)
    centres = []
    seg = None
    if crack is not None and crack.kind != CRACK_NONE:
        seg = (crack.x0 + 0.5, crack.x0 + crack.length - 0.5, crack.row + 0.5)
    tries = 0
    while fib.mean() < vf and tries < max_tries:
        tries += 1
        c = rng.uniform(0.0, 1.0, 2) * np.array([nx, ny])
        ok = True
        for q in centres:
            d = np.abs(c - q)
            d = np.minimum(d, np.array([nx, ny]) - d)
            if math.hypot(*d) < 2 * radius + gap:
                ok = False
                break
        if ok and seg is not None:
            # periodic distance from the centre to the crack segment
            best = np.inf
            for sx in (-nx, 0, nx):
                for sy in (-ny, 0, ny):
                    px, py = c[0] + sx, c[1] + sy
                    qx = min(max(px, seg[0]), seg[1])
                    best = min(best, math.hypot(px - qx, py - seg[2]))
            if best < radius + crack_clearance:
                ok = False
        if not ok:
            continue
        centres.append(c)
        fib |= _periodic_dist2(pts, c, (nx, ny)) <= radius * radius
    gid = fib.astype(np.int32)[None]
    C = [iso_constants(E_m, nu), iso_constants(E_f, nu)]
    m = _micro(n3, dim, gid, C, Gc=[Gc_m, Gc_f], crack=crack, name=name)
    m.fibre_centres = np.array(centres)
    return m


def inplane_rotations(n_grains, rng):
    th = rng.uniform(0.0, 2.0 * np.pi, n_grains)
    c, s = np.cos(th), np.sin(th)
    R = np.zeros((n_grains, 3, 3))
    R[:, 0, 0], R[:, 0, 1], R[:, 1, 0], R[:, 1, 1], R[:, 2, 2] = c, -s, s, c, 1.0
    return R


def so3_rotations(n_grains, rng):
    """Uniform random rotations from Shoemake's uniform unit quaternions."""
    u1, u2, u3 = rng.uniform(0.0, 1.0, (3, n_grains))
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    w, x, y, z = (b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                  a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3))
    R = np.empty((n_grains, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - z * w); R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w); R[:, 2, 1] = 2 * (y * z + x * w); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def voronoi(n, n_grains, seed, C=(1.0, 0.6, 0.5), orientation="inplane", Gc0=1.0, sigma_Gc=0.0,
            beta=0.0, cleave=(1.0, 0.0, 0.0), crack=None, name="voronoi"):
    """Periodic Voronoi polycrystal with uniform seeds (minimum-image distance), cubic grains.

    ``orientation`` is 'inplane' (uniform angle about z) or 'so3' (uniform on SO(3)). Local
    toughness is Gc0, or lognormal per grain, Gc0 * exp(sigma z - sigma^2 / 2), when sigma_Gc > 0.
    """
    from scipy.spatial import cKDTree

    n3, dim = _grid(n)
    nx, ny, nz = n3
    rng = np.random.default_rng(seed)
    box = np.array([nx, ny, nz], np.float64)[:dim]
    seeds = rng.uniform(0.0, 1.0, (n_grains, dim)) * box
    tree = cKDTree(seeds, boxsize=box)
    axes = [np.arange(v) + 0.5 for v in (nx, ny, nz)[:dim]]
    grids = np.meshgrid(*axes[::-1], indexing="ij")          # (z,) y, x order
    pts = np.stack(grids[::-1], -1).reshape(-1, dim)
    _, gid = tree.query(pts, k=1)
    gid = gid.reshape((nz, ny, nx)).astype(np.int32)
    R = inplane_rotations(n_grains, rng) if orientation == "inplane" else so3_rotations(n_grains, rng)
    if sigma_Gc > 0:
        Gc = Gc0 * np.exp(sigma_Gc * rng.standard_normal(n_grains) - 0.5 * sigma_Gc ** 2)
    else:
        Gc = np.full(n_grains, Gc0)
    return _micro(n3, dim, gid, [C] * n_grains, R=R, Gc=Gc, cleave=[cleave] * n_grains,
                  beta=[beta] * n_grains, crack=crack, name=name)


def laguerre_ids(n, n_grains, seed, sigma_size=0.25):
    """Grain ids (ny, nx) of a periodic Laguerre (power-weighted Voronoi) tessellation.

    Seeds are uniform in the cell; seed i gets the radius r_i = r_mean exp(s z_i - s^2 / 2),
    z_i ~ N(0, 1), s = sigma_size, r_mean half the mean seed spacing, and a voxel centre x joins
    the grain minimising |x - x_i|^2 - r_i^2 (minimum-image distance). Lognormal radii give a
    lognormal grain-size spread; sigma_size = 0 is the plain Voronoi tessellation. Ties go to the
    lowest seed index. Returns (gid, seeds, radii).
    """
    nx, ny = n
    rng = np.random.default_rng(seed)
    seeds = rng.uniform(0.0, 1.0, (n_grains, 2)) * np.array([nx, ny], np.float64)
    r_mean = 0.5 * np.sqrt(nx * ny / n_grains)
    radii = r_mean * np.exp(sigma_size * rng.standard_normal(n_grains) - 0.5 * sigma_size ** 2)
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    best = np.full((ny, nx), np.inf)
    gid = np.zeros((ny, nx), np.int32)
    for i in range(n_grains):
        dx = np.abs(x - seeds[i, 0])
        dx = np.minimum(dx, nx - dx)
        dy = np.abs(y - seeds[i, 1])
        dy = np.minimum(dy, ny - dy)
        pd = dy[:, None] ** 2 + dx[None, :] ** 2 - radii[i] ** 2
        upd = pd < best
        best[upd] = pd[upd]
        gid[upd] = i
    return gid, seeds, radii, rng


def polycrystal_plate(n=(256, 128), n_grains=60, seed=5, zener=4.0, beta=2.0, sigma_size=0.25,
                      orientation="so3", Gc0=1.0, crack=None, name="polycrystal_plate"):
    """Polycrystal plate one voxel thick, (nx, ny, 1) with six strain components (Sec. 5).

    Laguerre grains (``laguerre_ids``) with orientations uniform on SO(3) (three Euler angles'
    worth) or about z ('inplane'); cubic stiffness with C1111 : C1122 = 24 : 8 and C1212 from the
    Zener ratio z = 2 C1212 / (C1111 - C1122) (Eq. (zener)), scaled to C1111 = 1; one cleavage
    plane with normal R e1 and contrast beta (Eq. (PFFani)). With nz = 1 the damage gradient has
    no z component, so A acts through the in-plane projection of the normal.
    """
    nx, ny = n
    gid, _, _, rng = laguerre_ids(n, n_grains, seed, sigma_size)
    c11, c12 = 1.0, 8.0 / 24.0
    C = (c11, c12, 0.5 * zener * (c11 - c12))
    R = so3_rotations(n_grains, rng) if orientation == "so3" else inplane_rotations(n_grains, rng)
    return _micro((nx, ny, 1), 3, gid.reshape(1, ny, nx), [C] * n_grains, R=R, Gc=np.full(n_grains, Gc0),
                  cleave=[(1.0, 0.0, 0.0)] * n_grains, beta=[beta] * n_grains, crack=crack, name=name)


def _dtau(kappa, gc_ref, a_g, n_inc):
    return kappa * gc_ref * a_g / n_inc


# ----------------------------------------------------------------------------------------------
# Workloads. Sizes and distributions follow the paper's examples (Sec. 5): a homogeneous plate
# with a crack-tip-enriched crack, a random fibre composite and Voronoi polycrystals.
# ----------------------------------------------------------------------------------------------

def homogeneous_plate_64(n_inc=100, split=1):
    """64x64 plane-strain plate, E=1, nu=0.3, Gc=1, ell=2, CTE crack of 16 voxels at mid-height."""
    crack = Crack(CRACK_CTE, row=32, x0=0, length=16, phi_M=0.8, stiffness=1e-6)
    m = homogeneous((64, 64), 1.0, 0.3, 1.0, crack=crack, name="homogeneous_plate_64")
    w = Workload(m, ell=2.0, k_res=1e-6, split=split, n_inc=n_inc, name="homogeneous_plate_64")
    w.dtau = _dtau(1.5, 1.0, w.A_g, n_inc)
    return w


def fibre_composite_512(n_inc=300, seed=1, precision="fp64", n=512, radius=20.0):
    """Fibre composite: discs r=20 at 30% voxel fraction, E_f/E_m=5, Gc_f/Gc_m=2, ell=3,
    central CTE crack of n/8 voxels."""
    a0 = n // 8
    crack = Crack(CRACK_CTE, row=n // 2, x0=n // 2 - a0 // 2, length=a0, phi_M=0.8, stiffness=1e-6)
    m = fibres((n, n), radius, 0.30, seed, 1.0, 5.0, 0.3, 1.0, 2.0, crack=crack,
               crack_clearance=3 * 3.0, name=f"fibre_composite_{n}")
    w = Workload(m, ell=3.0, k_res=1e-6, split=0, n_inc=n_inc, precision=precision,
                 name=f"fibre_composite_{n}")
    w.dtau = _dtau(1.5, 1.0, w.A_g, n_inc)
    return w


def polycrystal_1024(n_inc=400, seed=2, n=1024, n_grains=200, precision="fp32r"):
    """Periodic Voronoi polycrystal, cubic C11=1, C12=0.6, C44=0.5 (Zener 2.5), in-plane
    orientations, cleavage beta=2 (contrast 1+beta=3), ell=2, CTE crack of 0.1 Lx."""
    a0 = int(round(0.1 * n))
    crack = Crack(CRACK_CTE, row=n // 2, x0=0, length=a0, phi_M=0.8, stiffness=1e-6)
    m = voronoi((n, n), n_grains, seed, (1.0, 0.6, 0.5), "inplane", beta=2.0, crack=crack,
                name=f"polycrystal_{n}")
    w = Workload(m, ell=2.0, k_res=1e-6, split=0, n_inc=n_inc, precision=precision,
                 name=f"polycrystal_{n}")
    w.dtau = _dtau(1.5, 1.0, w.A_g, n_inc)
    return w


def polycrystal_3d(n, n_grains, seed, n_inc=100, sigma_Gc=0.3, precision="fp32r"):
    a0 = max(1, int(round(0.1 * n)))
    crack = Crack(CRACK_CTE, row=n // 2, x0=0, length=a0, phi_M=0.8, stiffness=1e-6)
    m = voronoi((n, n, n), n_grains, seed, (1.0, 0.6, 0.5), "so3", sigma_Gc=sigma_Gc, crack=crack,
                name=f"polycrystal3d_{n}")
    w = Workload(m, ell=2.0, k_res=1e-6, split=0, n_inc=n_inc, precision=precision,
                 name=f"polycrystal3d_{n}")
    w.dtau = _dtau(1.5, float(np.mean(m.Gc)), w.A_g, n_inc)
    return w


def polycrystal_plate_256(n_inc=200, seed=5, zener=4.0, beta=2.0, precision="fp64"):
    """The polycrystal plate of Sec. 5 at power-of-two size: 256 x 128 x 1 voxels, 60 Laguerre
    grains with lognormal size spread 0.25, SO(3) orientations, Zener ratio 4, cleavage beta = 2,
    ell = 2, CTE crack of 0.1 Lx at mid-height."""
    a0 = 26
    crack = Crack(CRACK_CTE, row=64, x0=0, length=a0, phi_M=0.8, stiffness=1e-6)
    m = polycrystal_plate((256, 128), 60, seed, zener, beta, crack=crack, name="polycrystal_plate_256")
    w = Workload(m, ell=2.0, k_res=1e-6, split=0, n_inc=n_inc, precision=precision, name="polycrystal_plate_256")
    w.dtau = _dtau(1.5, 1.0, w.A_g, n_inc)
    return w


def batched_3d_polycrystals(count=16, seed=3, sizes=(32, 64, 128), n_inc=100):
    """A seeded mix of 3D polycrystals, grids drawn from ``sizes``, 50-200 grains each."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        g = int(rng.integers(50, 201))
        out.append(polycrystal_3d(n, g, seed * 1000 + i, n_inc=n_inc))
    return out


def serving_stream(count=512, seed=4, rate=1.0, sizes2d=(64, 128, 256, 512, 1024),
                   sizes3d=(32, 64, 128), n_inc=100):
    """Poisson arrival times and a seeded request mix (2D/3D, fibre/polycrystal).

    Returns a list of (arrival_time, kind, n, seed). Microstructures are built lazily by the
    consumer with :func:`build_request` so that a long trace stays cheap to describe.
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    reqs = []
    for i in range(count):
        is3d = rng.uniform() < 0.5
        kind = "fibre" if rng.uniform() < 0.5 else "poly"
        n = int(rng.choice(sizes3d if is3d else sizes2d))
        reqs.append((float(t[i]), kind, ("3d" if is3d else "2d"), n, seed * 100000 + i))
    return reqs


def build_request(kind, dims, n, seed, n_inc=100):
    if dims == "3d":
        return polycrystal_3d(n, int(np.random.default_rng(seed).integers(50, 201)), seed, n_inc=n_inc)
    if kind == "fibre":
        w = fibre_composite_512(n_inc=n_inc, seed=seed, n=n, radius=n / 25.6)
        w.precision = "fp32r"
        return w
    return polycrystal_1024(n_inc=n_inc, seed=seed, n=n, n_grains=max(8, (200 * n * n) // (1024 * 1024)))


def serving_mix(count=24, seed=4, n_inc=15, n_total=100, sizes2d=(64, 128, 256), sizes3d=(32,)):
    """A seeded request mix for the serving path: half 2D / half 3D grids, fibre composites and
    polycrystals from the generators above (fibre radius n/25.6, 50-200 grains). Each request
    uses the dissipation increment of a ``n_total``-increment run (as the benchmark workloads do)
    and is served for its first ``n_inc`` increments (or until fracture)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        is3d = rng.uniform() < 0.5
        n = int(rng.choice(sizes3d if is3d else sizes2d))
        s = seed * 100000 + i
        if is3d:
            w = polycrystal_3d(n, int(rng.integers(50, 201)), s, n_inc=n_total)
        elif rng.uniform() < 0.5:
            w = fibre_composite_512(n_inc=n_total, seed=s, n=n, radius=n / 25.6)
        else:
            w = polycrystal_1024(n_inc=n_total, seed=s, n=n, n_grains=int(rng.integers(50, 201)))
        w.n_inc = n_inc
        out.append(w)
    return out


def small_cases():
    """Small seeded cases for parity tests (several FFT tiles, non-square grids)."""
    cases = {}
    crack = Crack(CRACK_CTE, row=16, x0=0, length=8, phi_M=0.8, stiffness=1e-6)
    w = Workload(homogeneous((32, 32), crack=crack), ell=2.0, split=0, n_inc=12, name="homog32")
    w.dtau = _dtau(1.5, 1.0, w.A_g, 24)
    cases["homog32"] = w
    crack = Crack(CRACK_CTE, row=8, x0=4, length=8, phi_M=0.8, stiffness=1e-6)
    m = fibres((64, 16), 4.0, 0.25, 7, crack=crack, crack_clearance=2.0, name="fibre64x16")
    w = Workload(m, ell=2.0, split=0, n_inc=8, name="fibre64x16")
    w.dtau = _dtau(1.5, 1.0, w.A_g, 24)
    cases["fibre64x16"] = w
    crack = Crack(CRACK_CTE, row=16, x0=0, length=6, phi_M=0.8, stiffness=1e-6)
    m = voronoi((32, 32), 9, 11, beta=2.0, crack=crack, name="poly32")
    w = Workload(m, ell=2.0, split=0, n_inc=8, name="poly32")
    w.dtau = _dtau(1.5, 1.0, w.A_g, 24)
    cases["poly32"] = w
    crack = Crack(CRACK_CTE, row=8, x0=0, length=4, phi_M=0.8, stiffness=1e-6)
    m = voronoi((16, 16, 8), 6, 13, orientation="so3", sigma_Gc=0.3, crack=crack, name="poly3d")
    w = Workload(m, ell=2.0, split=0, n_inc=6, name="poly3d16x16x8")
    w.dtau = _dtau(1.5, float(np.mean(m.Gc)), w.A_g, 24)
    cases["poly3d"] = w
    crack = Crack(CRACK_CTE, row=8, x0=0, length=4, phi_M=0.8, stiffness=1e-6)
    m = polycrystal_plate((32, 16), 8, 17, zener=4.0, beta=2.0, crack=crack, name="plate32x16")
    w = Workload(m, ell=2.0, split=0, n_inc=6, name="plate32x16x1")
    w.dtau = _dtau(1.5, 1.0, w.A_g, 24)
    cases["plate3d"] = w
    return cases


def replace(w, **kw):
    return dataclasses.replace(w, **kw)


def config_names():
    """Names of the seeded workload configurations in configs.json."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "configs.json")) as f:
        return list(json.load(f))


def load_config(name):
    """Build the workload(s) of a named configuration of configs.json: a generator of this module,
    its keyword arguments (seeds included) and the precision. Returns a Workload, or a list of
    them for the batched and serving configurations."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "configs.json")) as f:
        c = json.load(f)[name]
    out = globals()[c["generator"]](**c["kwargs"])
    for w in (out if isinstance(out, list) else [out]):
        w.precision = c["precision"]
    return out
