"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module holds no arithmetic of the transport method: it only lays out
phantoms (voxel densities and material ids), material compositions and beam
spot lists, with the shapes, sizes and value distributions of the workloads
named below.  Both the oracle and the CUDA library receive exactly these
arrays.

Workloads (all synthetic, generated from a seed; no dataset is involved):

* ``water100``  - 10^4 protons, 100 MeV pencil beam (point source, +z) into
  homogeneous water (1.0 g/cm^3, I = 75 eV), 40 x 40 x 120 mm at 1 mm.
* ``slab150``   - 10^6 protons, 150 MeV Gaussian beam (sigma 3 mm), 60 x 60 x
  200 mm at 0.5 mm; z-slabs water [0,40) mm, cortical-bone-like
  (1.85 g/cm^3) [40,60), lung-like (0.26 g/cm^3, soft-tissue composition)
  [60,100), water beyond.
* ``insert150`` - 150 MeV beam, sigma 3 mm, 80 x 80 x 200 mm at 1 mm, water
  with a bone-like half-space insert (x > 0, z in [30,80) mm) whose edge lies
  on the beam axis.
* ``plan2000``  - 2000 spots on a 5 mm lateral grid, energies U(70,200) MeV,
  weights lognormal(0, 0.7), histories proportional to weight (largest
  remainder, total 10^8), 200 x 200 x 300 mm at 1 mm, water with 30 random
  spheres (radius U(5,25) mm, density U(0.2,1.9) g/cm^3, tissue or bone).

The paper's own test geometries (Sec. 2.2.2: 20 cm water cube, slab and
insert phantoms with 1 mm voxels) inform these shapes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Mass fractions.  Water as stated for the homogeneous workload; the bone-like
# and tissue-like compositions are the ICRU Report 46 cortical bone and soft
# tissue fractions restricted to the listed elements (each side renormalises).
WATER = {"name": "water", "elements": [(1, 0.1119), (8, 0.8881)], "I_eV": 75.0}
BONE = {
    "name": "bone",
    "elements": [(1, 0.034), (6, 0.155), (7, 0.042), (8, 0.435), (15, 0.103), (20, 0.225)],
    "I_eV": 0.0,  # Bragg-additive
}
TISSUE = {
    "name": "tissue",
    "elements": [(1, 0.102), (6, 0.143), (7, 0.034), (8, 0.708)],
    "I_eV": 0.0,
}

SPOT_DTYPE = np.dtype(
    [
        ("E_MeV", "f8"),
        ("sigma_E_MeV", "f8"),
        ("x_mm", "f8"),
        ("y_mm", "f8"),
        ("z_mm", "f8"),
        ("ux", "f8"),
        ("uy", "f8"),
        ("uz", "f8"),
        ("sigma_xy_mm", "f8"),
        ("sigma_angle_rad", "f8"),
        ("n_hist", "u8"),
    ]
)


@dataclass
class Workload:
    name: str
    shape: tuple  # (nx, ny, nz)
    voxel_mm: tuple
    origin_mm: tuple
    density: np.ndarray  # float32, shape (nz, ny, nx): x fastest in memory
    material_id: np.ndarray  # uint8, same shape
    materials: list
    spots: np.ndarray  # SPOT_DTYPE
    seed: int = 0
    notes: dict = field(default_factory=dict)

    @property
    def n_voxels(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz

    @property
    def n_histories(self) -> int:
        return int(self.spots["n_hist"].sum())

    def with_histories(self, total: int) -> "Workload":
        """Same phantom and spots, histories rescaled to ``total`` (largest remainder)."""
        spots = self.spots.copy()
        spots["n_hist"] = largest_remainder(spots["n_hist"].astype(np.float64), total)
        return Workload(self.name, self.shape, self.voxel_mm, self.origin_mm, self.density,
                        self.material_id, self.materials, spots, self.seed, dict(self.notes))


def largest_remainder(weights: np.ndarray, total: int) -> np.ndarray:
    """Integer counts proportional to ``weights`` that sum to ``total``."""
    w = np.asarray(weights, dtype=np.float64)
    if w.sum() <= 0:
        raise ValueError("weights must have a positive sum")
    exact = w / w.sum() * total
    base = np.floor(exact).astype(np.uint64)
    rem = int(total - int(base.sum()))
    order = np.argsort(-(exact - base), kind="stable")
    base[order[:rem]] += 1
    return base


def pencil(E, n, x=0.0, y=0.0, z=0.0, sigma_xy=0.0, sigma_E=0.0, sigma_angle=0.0,
           u=(0.0, 0.0, 1.0)) -> np.ndarray:
    s = np.zeros(1, dtype=SPOT_DTYPE)
    s[0] = (E, sigma_E, x, y, z, u[0], u[1], u[2], sigma_xy, sigma_angle, n)
    return s


def _grid(nx, ny, nz, h):
    """Voxel-centre coordinates (mm) for a grid whose x/y are centred on 0 and z starts at 0."""
    ox, oy, oz = -nx * h / 2.0, -ny * h / 2.0, 0.0
    xc = ox + (np.arange(nx) + 0.5) * h
    yc = oy + (np.arange(ny) + 0.5) * h
    zc = oz + (np.arange(nz) + 0.5) * h
    return (ox, oy, oz), xc, yc, zc


def water100(n_hist: int = 10_000) -> Workload:
    nx, ny, nz, h = 40, 40, 120, 1.0
    origin, *_ = _grid(nx, ny, nz, h)
    dens = np.ones((nz, ny, nx), np.float32)
    mid = np.zeros((nz, ny, nx), np.uint8)
    return Workload("water100", (nx, ny, nz), (h, h, h), origin, dens, mid, [WATER],
                    pencil(100.0, n_hist), seed=0)


def slab150(n_hist: int = 1_000_000) -> Workload:
    nx, ny, nz, h = 120, 120, 400, 0.5
    origin, xc, yc, zc = _grid(nx, ny, nz, h)
    dens = np.ones((nz, ny, nx), np.float32)
    mid = np.zeros((nz, ny, nx), np.uint8)
    bone = (zc >= 40) & (zc < 60)
    lung = (zc >= 60) & (zc < 100)
    dens[bone] = 1.85
    mid[bone] = 1
    dens[lung] = 0.26
    mid[lung] = 2
    return Workload("slab150", (nx, ny, nz), (h, h, h), origin, dens, mid, [WATER, BONE, TISSUE],
                    pencil(150.0, n_hist, sigma_xy=3.0), seed=0)


def insert150(n_hist: int = 10_000_000) -> Workload:
    nx, ny, nz, h = 80, 80, 200, 1.0
    origin, xc, yc, zc = _grid(nx, ny, nz, h)
    dens = np.ones((nz, ny, nx), np.float32)
    mid = np.zeros((nz, ny, nx), np.uint8)
    ins = ((zc >= 30) & (zc < 80))[:, None, None] & (xc > 0)[None, None, :]
    ins = np.broadcast_to(ins, dens.shape)
    dens[ins] = 1.85
    mid[ins] = 1
    return Workload("insert150", (nx, ny, nz), (h, h, h), origin, dens, mid, [WATER, BONE],
                    pencil(150.0, n_hist, sigma_xy=3.0), seed=0,
                    notes={"profile_depths_mm": [20.0, 50.0, 90.0]})


def sphere_phantom(shape, h, seed, n_spheres=30, r_range=(5.0, 25.0), rho_range=(0.2, 1.9)):
    """Water with random spherical inserts; later spheres overwrite earlier ones.

    Material ids: 0 water, 1 tissue-like, 2 bone-like.  Each sphere is drawn as
    (radius, centre, density, composition) and rasterised by voxel-centre inclusion.
    """
    nx, ny, nz = shape
    origin, xc, yc, zc = _grid(nx, ny, nz, h)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5DE]))
    dens = np.ones((nz, ny, nx), np.float32)
    mid = np.zeros((nz, ny, nx), np.uint8)
    ext = np.array([nx * h, ny * h, nz * h])
    lo = np.array(origin)
    for _ in range(n_spheres):
        r = rng.uniform(*r_range)
        c = lo + rng.uniform(0.0, 1.0, 3) * ext
        rho = rng.uniform(*rho_range)
        m = 2 if rng.uniform() < 0.5 else 1
        # only the voxels of the sphere's bounding box can be inside it
        ix = np.nonzero(np.abs(xc - c[0]) <= r)[0]
        iy = np.nonzero(np.abs(yc - c[1]) <= r)[0]
        iz = np.nonzero(np.abs(zc - c[2]) <= r)[0]
        if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
            continue
        Z, Y, X = np.meshgrid(zc[iz], yc[iy], xc[ix], indexing="ij")
        inside = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= r * r
        sub = np.ix_(iz, iy, ix)
        dsub = dens[sub]
        msub = mid[sub]
        dsub[inside] = rho
        msub[inside] = m
        dens[sub] = dsub
        mid[sub] = msub
    return origin, dens, mid


def plan_spots(n_spots, total, seed, e_range=(70.0, 200.0), pitch=5.0, half_width=100.0):
    """Spots on a ``pitch`` lateral grid inside +-half_width, energies uniform, weights
    lognormal(0, 0.7), histories by largest remainder.  When there are more spots than
    grid points the positions repeat (several energy layers share a position)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5B07]))
    g = np.arange(-half_width + pitch / 2.0, half_width, pitch)
    gx, gy = np.meshgrid(g, g, indexing="xy")
    pts = np.stack([gx.ravel(), gy.ravel()], 1)
    order = rng.permutation(len(pts))
    pos = pts[np.resize(order, n_spots)]
    E = rng.uniform(*e_range, n_spots)
    w = rng.lognormal(0.0, 0.7, n_spots)
    spots = np.zeros(n_spots, SPOT_DTYPE)
    spots["E_MeV"] = E
    spots["x_mm"] = pos[:, 0]
    spots["y_mm"] = pos[:, 1]
    spots["uz"] = 1.0
    spots["n_hist"] = largest_remainder(w, total)
    return spots


def plan2000(total: int = 100_000_000, seed: int = 0) -> Workload:
    nx, ny, nz, h = 200, 200, 300, 1.0
    origin, dens, mid = sphere_phantom((nx, ny, nz), h, seed)
    spots = plan_spots(2000, total, seed)
    return Workload("plan2000", (nx, ny, nz), (h, h, h), origin, dens, mid, [WATER, TISSUE, BONE],
                    spots, seed=seed)


def denoise_case(seed: int, n_hist: int = 100_000, shape=(128, 128, 192), n_spots: int = 24,
                 sigma_xy_mm: float = 3.0) -> Workload:
    """One sample of the denoiser workload: 128 x 128 x 192 mm at 1 mm, water with 30
    random spheres (radius 5-15 mm, density 0.2-1.9, tissue or bone) and a plan of
    ``n_spots`` Gaussian spots (sigma ``sigma_xy_mm``, as the slab and insert beams) on
    a 5 mm lateral grid within +-30 mm, energies U(70, 200) MeV (ranges beyond the
    phantom exit), weights lognormal(0, 0.7), ``n_hist`` protons."""
    nx, ny, nz = shape
    origin, dens, mid = sphere_phantom(shape, 1.0, seed, r_range=(5.0, 15.0))
    spots = plan_spots(n_spots, n_hist, seed, pitch=5.0, half_width=30.0)
    spots["sigma_xy_mm"] = sigma_xy_mm
    return Workload(f"denoise{seed}", shape, (1.0, 1.0, 1.0), origin, dens, mid, [WATER, TISSUE, BONE], spots,
                    seed=seed)


WORKLOADS = {"water100": water100, "slab150": slab150, "insert150": insert150,
             "plan2000": plan2000, "denoise_case": denoise_case}
