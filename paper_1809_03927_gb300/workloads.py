"""Seeded synthetic inputs: HU phantoms, spot plans and deformation fields.

This module only draws and lays out inputs.  It holds none of the dose
method's arithmetic (no calibration, physics, timeline or accumulation), so
both the CUDA path's tests/benchmark and the CPU oracle may use it.

The paper's patient data (Table I: lung, esophagus and liver 4DCTs of
427x246x161 to 452x307x281 voxels, 2-3 fields) is not available; these
phantoms stand in for it with comparable sizes and structure:

* ``water_phantom``   homogeneous water, one pencil beam (the single-spot case)
* ``slab_phantom``    water / lung / bone slabs, 400 spots on 10 layers
* ``phantom_4dct``    body, two lungs and a tumour moving sinusoidally in the
                      superior-inferior direction over N breathing phases, with
                      the matching displacement fields to phase 0 (Sec. 2.A:
                      4DCT sorted into N = 10 phases; Sec. 2.D.1: DVFs map each
                      phase onto the accumulation phase)
* ``random_phantom``  random slabs and spheres for ragged job batches

Grids are ``int16`` HU arrays of shape ``(nz, ny, nx)`` (x fastest).  A grid
voxel ``(i, j, k)`` covers ``[i dx, (i+1) dx) x [j dy, ...) x [k dz, ...)`` in
grid millimetres; ``origin`` is the patient-frame position of the grid corner.
Spot lateral coordinates are patient-frame millimetres on the two axes other
than the beam axis, lower axis first.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

HU_AIR, HU_WATER, HU_LUNG_SLAB, HU_BONE, HU_LUNG, HU_TUMOUR = -1000, 0, -740, 1200, -800, 40


@dataclass
class Phantom:
    hu: np.ndarray                    # (nz, ny, nx) int16, or (P, nz, ny, nx)
    d: tuple                          # voxel size (dx, dy, dz), mm
    origin: tuple                     # patient-frame mm of the grid corner
    beam_axis: int = 2                # 0 = x, 1 = y, 2 = z
    beam_sign: int = 1

    @property
    def n(self):
        s = self.hu.shape
        return (s[-1], s[-2], s[-3])

    @property
    def n_phases(self):
        return 1 if self.hu.ndim == 3 else self.hu.shape[0]

    @property
    def beam_dir(self):
        v = [0.0, 0.0, 0.0]
        v[self.beam_axis] = float(self.beam_sign)
        return tuple(v)


@dataclass
class Plan:
    x: np.ndarray                     # float64 (n,)
    y: np.ndarray
    energy: np.ndarray                # MeV
    sigma: np.ndarray                 # mm
    protons: np.ndarray               # uint64
    layer: np.ndarray                 # int32
    field: np.ndarray                 # int32

    def __len__(self):
        return int(self.x.shape[0])

    def subset(self, idx):
        idx = np.asarray(idx)
        return Plan(self.x[idx], self.y[idx], self.energy[idx], self.sigma[idx],
                    self.protons[idx], self.layer[idx], self.field[idx])

    def with_protons(self, protons):
        return Plan(self.x, self.y, self.energy, self.sigma,
                    np.asarray(protons, dtype=np.uint64), self.layer, self.field)


@dataclass
class Delivery:
    """Delivery-clock inputs (Sec. 2.B, App. A), integer nanoseconds."""
    n_phases: int = 10
    start_phase: int = -1             # -1: drawn from the seed
    gated: int = 0
    gate_first: int = 0
    gate_last: int = 0
    repaints: int = 1
    period_ns: int = 4_000_000_000
    period_sigma_ns: int = 0
    spot_switch_ns: int = 2_000_000
    layer_switch_ns: int = 1_000_000_000
    discard_ns: int = 0
    rate_protons_per_s: int = 1_000_000_000
    seed: int = 3
    synchrotron: int = 0              # 1: fills with charge / extraction-time limits (App. A)
    reserved: int = 0
    fill_protons: int = 0             # protons per synchrotron fill (0: unlimited)
    extraction_limit_ns: int = 0      # extraction time per fill (0: unlimited)
    max_protons_per_paint: int = 0    # isolayered repainting cap per spot (0: off)


@dataclass
class DeliverySpread:
    """Spread of the delivery parameters over uncertainty trials (Sec. 2.B):
    the breathing period from a discrete uniform set, the synchrotron
    parameters Gaussian about the delivery's values."""
    period_min_ns: int = 0
    period_max_ns: int = 0
    period_step_ns: int = 0
    spot_switch_sigma_ns: int = 0
    layer_switch_sigma_ns: int = 0
    discard_sigma_ns: int = 0
    rate_sigma: int = 0
    fill_protons_sigma: int = 0
    extraction_limit_sigma_ns: int = 0


def _plan(xs, ys, es, sig, protons, layers, fields):
    return Plan(np.asarray(xs, np.float64), np.asarray(ys, np.float64),
                np.asarray(es, np.float64), np.asarray(sig, np.float64),
                np.asarray(protons, np.uint64), np.asarray(layers, np.int32),
                np.asarray(fields, np.int32))


# --------------------------------------------------------------------------
# single pencil beam in water
# --------------------------------------------------------------------------
def water_phantom(nx=64, ny=64, nz=160, d=2.0, hu=HU_WATER):
    """Homogeneous phantom, beam along +z entering at the lateral centre."""
    vol = np.full((nz, ny, nx), hu, dtype=np.int16)
    return Phantom(vol, (d, d, d), (-nx * d / 2.0, -ny * d / 2.0, 0.0), 2, 1)


def pencil_plan(energy=150.0, sigma=4.0, protons=1_000_000, x=0.0, y=0.0):
    return _plan([x], [y], [energy], [sigma], [protons], [0], [0])


# --------------------------------------------------------------------------
# heterogeneous slab phantom, 400 spots on 10 layers
# --------------------------------------------------------------------------
def slab_phantom(n=128, d=2.0, slabs=((20.0, HU_WATER), (40.0, HU_LUNG_SLAB), (10.0, HU_BONE))):
    """Slabs stacked along +z from the entry face, water after the last."""
    vol = np.full((n, n, n), HU_WATER, dtype=np.int16)
    z = (np.arange(n) + 0.5) * d
    top = 0.0
    for thick, hu in slabs:
        sel = (z >= top) & (z < top + thick)
        vol[sel, :, :] = hu
        top += thick
    return Phantom(vol, (d, d, d), (-n * d / 2.0, -n * d / 2.0, 0.0), 2, 1)


def slab_plan(seed=2, n_layers=10, e_lo=70.0, e_hi=200.0, nx=8, ny=5, pitch=5.0,
              sigma=4.0, w_lo=0.5e6, w_hi=1.5e6):
    """``nx x ny`` spots per layer on a ``pitch`` grid centred on the axis;
    layers delivered from the highest energy down; weights U[w_lo, w_hi]."""
    rng = np.random.default_rng(seed)
    energies = np.linspace(e_lo, e_hi, n_layers)[::-1]
    gx = (np.arange(nx) - (nx - 1) / 2.0) * pitch
    gy = (np.arange(ny) - (ny - 1) / 2.0) * pitch
    xs, ys, es, ls = [], [], [], []
    for li, e in enumerate(energies):
        for j, yv in enumerate(gy):
            row = gx if j % 2 == 0 else gx[::-1]          # serpentine scan
            for xv in row:
                xs.append(xv); ys.append(yv); es.append(e); ls.append(li)
    n = len(xs)
    w = np.floor(rng.uniform(w_lo, w_hi, size=n)).astype(np.uint64)
    return _plan(xs, ys, es, [sigma] * n, w, ls, [0] * n)


# --------------------------------------------------------------------------
# synthetic 4DCT with moving tumour and DVFs to phase 0
# --------------------------------------------------------------------------
@dataclass
class Geometry4D:
    centre: tuple                       # body axis (x, y) in grid mm
    body_axes: tuple                    # elliptic-cylinder semi-axes (x, y)
    lungs: list                         # [(centre xyz, semi-axes xyz)]
    tumour_centre0: tuple               # grid mm, phase-0 centre of motion
    tumour_radius: float
    amplitude: float                    # half of the peak-to-peak motion
    n_phases: int
    taper: float = 10.0

    def tumour_z(self, p):
        """Superior-inferior tumour position of phase p (sinusoidal motion)."""
        return self.tumour_centre0[2] + self.amplitude * np.cos(2.0 * np.pi * p / self.n_phases)


def _grid_centres(n, d):
    nx, ny, nz = n
    x = (np.arange(nx, dtype=np.float64) + 0.5) * d[0]
    y = (np.arange(ny, dtype=np.float64) + 0.5) * d[1]
    z = (np.arange(nz, dtype=np.float64) + 0.5) * d[2]
    return x, y, z


def _ellipsoid_r(x, y, z, c, a):
    return np.sqrt(((x - c[0]) / a[0]) ** 2 + ((y - c[1]) / a[1]) ** 2 + ((z - c[2]) / a[2]) ** 2)


def phantom_4dct(nx=256, ny=256, nz=160, d=(1.0, 1.0, 2.5), n_phases=10,
                 motion_pp=15.0, tumour_diameter=30.0, with_dvf=True):
    """Body (water) in air, two lungs (-800 HU), a tumour sphere (+40 HU) in
    the right lung moving sinusoidally along z with ``motion_pp`` peak to
    peak; beam along +y (anterior-posterior).

    Returns ``(phantom, dvf, geometry)``: ``dvf`` is float32 of shape
    ``(P, 3, nz, ny, nx)`` in mm, the displacement that carries each phase-p
    point onto phase 0, sampled at voxel centres (zero for phase 0).
    Geometry scales with the grid extent so that small grids keep the same
    layout.
    """
    ext = (nx * d[0], ny * d[1], nz * d[2])
    cx, cy = ext[0] / 2.0, ext[1] / 2.0
    sx, sy = ext[0] / 256.0, ext[1] / 256.0
    sz = ext[2] / 400.0
    body = (120.0 * sx, 90.0 * sy)
    lung_axes = (40.0 * sx, 55.0 * sy, 110.0 * sz)
    lungs = [((cx - 55.0 * sx, cy - 8.0 * sy, ext[2] / 2.0), lung_axes),
             ((cx + 55.0 * sx, cy - 8.0 * sy, ext[2] / 2.0), lung_axes)]
    geo = Geometry4D((cx, cy), body, lungs, (cx - 55.0 * sx, cy - 8.0 * sy, ext[2] / 2.0),
                     tumour_diameter / 2.0 * min(1.0, sx, sy), motion_pp / 2.0, n_phases)
    x, y, z = _grid_centres((nx, ny, nz), d)
    X = x[None, None, :]
    Y = y[None, :, None]
    Z = z[:, None, None]
    in_body = (((X - cx) / body[0]) ** 2 + ((Y - cy) / body[1]) ** 2) <= 1.0
    in_lung = np.zeros((nz, ny, nx), dtype=bool)
    lung_r = np.full((nz, ny, nx), np.inf)
    for c, a in lungs:
        r = _ellipsoid_r(X, Y, Z, c, a)
        in_lung |= r <= 1.0
        lung_r = np.minimum(lung_r, r)
    base = np.where(in_body, HU_WATER, HU_AIR).astype(np.int16)
    base = np.where(in_lung & in_body, HU_LUNG, base).astype(np.int16)
    hu = np.empty((n_phases, nz, ny, nx), dtype=np.int16)
    # moving-region weight m: 1 inside the lungs, tapered to 0 over `taper` mm
    # outside (distance approximated along the scaled radius)
    amin = min(lung_axes)
    m = np.clip(1.0 - (lung_r - 1.0) * amin / geo.taper, 0.0, 1.0)
    m = np.where(in_body, m, 0.0)
    dvf = np.zeros((n_phases, 3, nz, ny, nx), dtype=np.float32) if with_dvf else None
    z0 = geo.tumour_z(0)
    for p in range(n_phases):
        zc = geo.tumour_z(p)
        vol = base.copy()
        rt = np.sqrt((X - geo.tumour_centre0[0]) ** 2 + (Y - geo.tumour_centre0[1]) ** 2 + (Z - zc) ** 2)
        vol[rt <= geo.tumour_radius] = HU_TUMOUR
        hu[p] = vol
        if with_dvf and p > 0:
            dvf[p, 2] = (-(zc - z0) * m).astype(np.float32)
    ph = Phantom(hu, tuple(float(v) for v in d), (-cx, -cy, 0.0), 1, 1)
    return ph, dvf, geo


def reference_to_phase_field(dvf):
    """The dose-interpolation method pulls dose and needs the field in the
    other direction from the one ``phantom_4dct`` returns: the displacement
    carrying a phase-0 (reference) point to phase p, given at the reference
    voxel centres.  The breathing model moves points along z by the same
    weight map m(r) in both images, so that field is the negated one (like
    the fields of a registration run in each direction, the two are not
    exact inverses where m varies)."""
    return None if dvf is None else (-dvf).astype(np.float32)


def tumour_plan(geo: Geometry4D, origin, seed=3, n_layers=20, per_layer=150,
                e_lo=70.0, e_hi=180.0, pitch=5.0, sigma=4.0, w_lo=0.5e6, w_hi=1.5e6):
    """AP plan over the tumour and its motion: on each of ``n_layers`` layers
    (highest energy first) the ``per_layer`` points of a ``pitch`` square grid
    nearest the tumour's mean position (a disc), scanned row by row in a
    serpentine.  Lateral axes of an AP beam are (x, z)."""
    rng = np.random.default_rng(seed)
    cx = geo.tumour_centre0[0] + origin[0]
    cz = geo.tumour_centre0[2] + origin[2]
    half = int(np.ceil(np.sqrt(per_layer))) + 2
    pts = []
    for j in range(-half, half + 1):
        for i in range(-half, half + 1):
            pts.append((i * pitch, j * pitch))
    pts = np.array(pts)
    dist = np.hypot(pts[:, 0], pts[:, 1])
    order = np.lexsort((np.arange(len(pts)), dist))[:per_layer]
    sel = pts[order]
    # serpentine ordering of the selected disc points: by row, alternating
    rows = sorted(set(sel[:, 1]))
    scan = []
    for r_i, rv in enumerate(rows):
        row = sorted([p for p in sel if p[1] == rv], key=lambda p: p[0])
        if r_i % 2:
            row = row[::-1]
        scan.extend(row)
    scan = np.array(scan)
    energies = np.linspace(e_lo, e_hi, n_layers)[::-1]
    xs, ys, es, ls = [], [], [], []
    for li, e in enumerate(energies):
        for px, pz in scan:
            xs.append(cx + px); ys.append(cz + pz); es.append(e); ls.append(li)
    n = len(xs)
    w = np.floor(rng.uniform(w_lo, w_hi, size=n)).astype(np.uint64)
    return _plan(xs, ys, es, [sigma] * n, w, ls, [0] * n)


# --------------------------------------------------------------------------
# random phantoms and plans for ragged job batches
# --------------------------------------------------------------------------
def random_phantom(rng, side, d=2.0):
    """Cube of ``side`` voxels: water with 1-3 random slabs and 0-3 spheres."""
    vol = np.full((side, side, side), HU_WATER, dtype=np.int16)
    ext = side * d
    z = (np.arange(side) + 0.5) * d
    for _ in range(int(rng.integers(1, 4))):
        z0 = rng.uniform(0.0, ext * 0.8)
        th = rng.uniform(5.0, 40.0)
        hu = int(rng.choice([HU_LUNG_SLAB, HU_BONE, -300, 200]))
        vol[(z >= z0) & (z < z0 + th)] = hu
    x = (np.arange(side) + 0.5) * d
    X = x[None, None, :]; Y = x[None, :, None]; Z = z[:, None, None]
    for _ in range(int(rng.integers(0, 4))):
        c = rng.uniform(0.2 * ext, 0.8 * ext, size=3)
        r = rng.uniform(5.0, 25.0)
        hu = int(rng.choice([HU_LUNG, HU_BONE, HU_TUMOUR, -500]))
        vol[((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) <= r * r] = hu
    return Phantom(vol, (d, d, d), (-ext / 2.0, -ext / 2.0, 0.0), 2, 1)


def random_plan(rng, n_spots, half_width, e_lo=70.0, e_hi=220.0, sigma=4.0):
    """``n_spots`` spots uniform over a square of ``half_width`` mm, energies
    U[e_lo, e_hi] grouped into layers of equal energy, weights U[0.5,1.5]e6."""
    n_layers = max(1, min(20, n_spots // 20))
    layer_e = np.sort(rng.uniform(e_lo, e_hi, size=n_layers))[::-1]
    layer = np.sort(rng.integers(0, n_layers, size=n_spots)).astype(np.int32)
    xs = rng.uniform(-half_width, half_width, size=n_spots)
    ys = rng.uniform(-half_width, half_width, size=n_spots)
    w = np.floor(rng.uniform(0.5e6, 1.5e6, size=n_spots)).astype(np.uint64)
    return _plan(xs, ys, layer_e[layer], np.full(n_spots, sigma), w, layer, np.zeros(n_spots))


def log_uniform_int(rng, lo, hi):
    return int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))
