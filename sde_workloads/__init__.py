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

* ``ct_sobp``    - thorax-like synthetic CT, 120 x 120 x 240 mm at 1 mm (HU -> density by
  a piecewise-linear calibration, HU bins -> air / lung / adipose / soft tissue /
  cortical bone), spread-out Bragg peak of 16 layers (ranges 90-140 mm in water).
* ``sobp_water`` - the same spread-out Bragg peak in water.

The paper's own test geometries (Sec. 2.2.2: 20 cm water cube, slab and
insert phantoms with 1 mm voxels) inform these shapes; its conclusion names patient
CT geometries and spread-out Bragg peaks as the next validation step.
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


# ---------------------------------------------------------------------------
# CT-like phantoms and spread-out Bragg peaks (synthetic; no patient data).
# Tissue compositions: ICRU Report 44 mass fractions, restricted to elements above
# 0.1 % (each side renormalises); air: dry air at sea level.
AIR = {"name": "air", "elements": [(6, 0.000124), (7, 0.755268), (8, 0.231781), (18, 0.012827)],
       "I_eV": 85.7}
LUNG = {"name": "lung", "elements": [(1, 0.103), (6, 0.105), (7, 0.031), (8, 0.749), (11, 0.002), (15, 0.002),
                                     (16, 0.003), (17, 0.003), (19, 0.002)], "I_eV": 0.0}
ADIPOSE = {"name": "adipose", "elements": [(1, 0.114), (6, 0.598), (7, 0.007), (8, 0.278), (11, 0.001),
                                           (16, 0.001), (17, 0.001)], "I_eV": 0.0}
SOFT = {"name": "soft tissue", "elements": [(1, 0.102), (6, 0.143), (7, 0.034), (8, 0.708), (11, 0.002),
                                            (15, 0.003), (16, 0.003), (17, 0.002), (19, 0.003)], "I_eV": 0.0}
CORTICAL = {"name": "cortical bone", "elements": [(1, 0.034), (6, 0.155), (7, 0.042), (8, 0.435), (11, 0.001),
                                                  (12, 0.002), (15, 0.103), (16, 0.003), (20, 0.225)], "I_eV": 0.0}
CT_MATERIALS = [AIR, LUNG, ADIPOSE, SOFT, CORTICAL]
# upper HU bound of each material bin (air < -900 <= lung < -200 <= adipose < -30 <= soft < 150 <= bone)
CT_HU_BINS = (-900.0, -200.0, -30.0, 150.0)


def hu_to_density(hu):
    """Piecewise-linear CT calibration (g/cm^3): 1 + HU/1000 below water (air at -1000,
    floored at 0.0012) and 1 + 0.00058 HU above it (cortical bone ~1.9 at 1500 HU)."""
    hu = np.asarray(hu, dtype=np.float64)
    rho = np.where(hu <= 0.0, 1.0 + hu / 1000.0, 1.0 + 0.00058 * hu)
    return np.maximum(rho, 0.0012).astype(np.float32)


def hu_to_material(hu):
    """Material id by HU bin (index into CT_MATERIALS)."""
    return np.searchsorted(np.asarray(CT_HU_BINS), np.asarray(hu, dtype=np.float64), side="right").astype(np.uint8)


def thorax_hu(shape=(120, 120, 240), h=1.0, seed=0):
    """A thorax-like HU volume (nz, ny, nx), beam axis along +z: an elliptic body (adipose
    shell 6 mm, soft tissue), two lungs with an airway between them, a rib layer in
    front of the lungs, a spine behind the mediastinum, air outside and in front of the
    skin; HU noise sigma 12 (seeded)."""
    nx, ny, nz = shape
    _, xc, yc, zc = _grid(nx, ny, nz, h)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xC7]))
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    hu = np.full((nz, ny, nx), -1000.0)
    zb0, zb1 = 8.0, nz * h - 8.0                      # body extent along the beam
    rx, ry = 0.47 * nx * h, 0.45 * ny * h             # body ellipse (x-y)
    body = ((X / rx) ** 2 + (Y / ry) ** 2 <= 1.0) & (Z >= zb0) & (Z < zb1)
    hu[body] = 40.0
    skin = body & (((X / (rx - 6)) ** 2 + (Y / (ry - 6)) ** 2 > 1.0) | (Z < zb0 + 6) | (Z >= zb1 - 6))
    hu[skin] = -90.0
    ribs = body & (Z >= zb0 + 14) & (Z < zb0 + 22) & (np.abs(np.sin(Y / 6.0)) > 0.3)
    hu[ribs] = 800.0
    for sx in (-1.0, 1.0):                             # lungs
        lung = body & (((X - sx * 0.22 * nx * h) / (0.18 * nx * h)) ** 2 + (Y / (0.33 * ny * h)) ** 2 +
                       ((Z - 0.45 * nz * h) / (0.25 * nz * h)) ** 2 <= 1.0)
        hu[lung] = -780.0
    airway = body & (X ** 2 + (Y - 0.05 * ny * h) ** 2 <= 7.0 ** 2) & (Z >= 0.3 * nz * h) & (Z < 0.6 * nz * h)
    hu[airway] = -980.0
    spine = body & (X ** 2 + ((Y + 0.0 * ny * h) ** 2) <= 14.0 ** 2) & (Z >= 0.7 * nz * h) & (Z < 0.85 * nz * h)
    hu[spine] = 1100.0
    tumour = body & ((X - 0.2 * nx * h) ** 2 + Y ** 2 + (Z - 0.42 * nz * h) ** 2 <= 12.0 ** 2)
    hu[tumour] = 45.0
    hu[body] += rng.normal(0.0, 12.0, int(body.sum()))
    return hu


def bragg_kleeman_energy(range_mm, alpha=0.0022, p=1.77):
    """Energy (MeV) whose CSDA range in water is range_mm by the Bragg-Kleeman rule
    R = alpha E^p (R in cm)."""
    return (np.asarray(range_mm, dtype=np.float64) / 10.0 / alpha) ** (1.0 / p)


def sobp_layer_weights(r_lo_mm, r_hi_mm, n_layers, p=1.77):
    """Relative fluence of n equally spaced range layers for a flat spread-out Bragg peak
    over [r_lo, r_hi] (Bortfeld & Schlegel 1996): with pristine curves ~ (R - z)^(1/p - 1)
    the flat superposition has weight density w(R) ~ (R_max - R)^(-1/p); each layer gets
    the integral of w over its range bin (the deepest bin ends at R_max)."""
    R = np.linspace(r_lo_mm, r_hi_mm, n_layers)
    dR = (r_hi_mm - r_lo_mm) / (n_layers - 1)
    lo = np.maximum(R - dR / 2.0, r_lo_mm - dR / 2.0)
    hi = np.minimum(R + dR / 2.0, r_hi_mm)
    q = 1.0 - 1.0 / p
    w = ((r_hi_mm - lo) ** q - (r_hi_mm - hi) ** q) / q
    return R, w / w.sum()


def sobp_spots(total, r_lo_mm, r_hi_mm, n_layers=16, x_mm=0.0, y_mm=0.0, half_width_mm=10.0, pitch_mm=5.0,
               sigma_xy_mm=3.0, energy_spread=0.008):
    """A spread-out Bragg peak: n_layers energies (Bragg-Kleeman) for ranges r_lo..r_hi in
    water, spaced closer than a pristine peak's width, energy spread 0.8 % (sigma), layer
    fluences by the Bortfeld-Schlegel weighting, each layer a square grid of Gaussian
    spots (sigma_xy) of side 2 half_width centred on (x, y); histories by largest
    remainder."""
    R, w = sobp_layer_weights(r_lo_mm, r_hi_mm, n_layers)
    E = bragg_kleeman_energy(R)
    g = np.arange(-half_width_mm + pitch_mm / 2.0, half_width_mm, pitch_mm)
    gx, gy = np.meshgrid(g, g, indexing="xy")
    n_grid = gx.size
    spots = np.zeros(n_layers * n_grid, SPOT_DTYPE)
    spots["E_MeV"] = np.repeat(E, n_grid)
    spots["sigma_E_MeV"] = energy_spread * spots["E_MeV"]
    spots["x_mm"] = np.tile(gx.ravel(), n_layers) + x_mm
    spots["y_mm"] = np.tile(gy.ravel(), n_layers) + y_mm
    spots["uz"] = 1.0
    spots["sigma_xy_mm"] = sigma_xy_mm
    spots["n_hist"] = largest_remainder(np.repeat(w / n_grid, n_grid), total)
    return spots


def ct_sobp(n_hist: int = 1_000_000, seed: int = 0, shape=(120, 120, 240), h: float = 1.0) -> Workload:
    """Thorax-like CT phantom (HU -> density and one of five ICRU 44 materials) irradiated by
    a spread-out Bragg peak, 16 layers covering ranges 90-140 mm in water, 20 x 20 mm
    field of 5 mm-spaced Gaussian spots aimed at the tumour insert."""
    nx, ny, nz = shape
    origin, *_ = _grid(nx, ny, nz, h)
    hu = thorax_hu(shape, h, seed)
    spots = sobp_spots(n_hist, 90.0, 140.0, x_mm=0.2 * nx * h)
    return Workload(f"ct_sobp{seed}", shape, (h, h, h), origin, hu_to_density(hu), hu_to_material(hu),
                    list(CT_MATERIALS), spots, seed=seed, notes={"hu": hu})


def sobp_water(n_hist: int = 1_000_000) -> Workload:
    """The same spread-out Bragg peak in water (80 x 80 x 200 mm at 1 mm), for its flatness."""
    nx, ny, nz, h = 80, 80, 200, 1.0
    origin, *_ = _grid(nx, ny, nz, h)
    return Workload("sobp_water", (nx, ny, nz), (h, h, h), origin, np.ones((nz, ny, nx), np.float32),
                    np.zeros((nz, ny, nx), np.uint8), [WATER], sobp_spots(n_hist, 90.0, 140.0))


WORKLOADS = {"water100": water100, "slab150": slab150, "insert150": insert150,
             "plan2000": plan2000, "denoise_case": denoise_case, "ct_sobp": ct_sobp, "sobp_water": sobp_water}
