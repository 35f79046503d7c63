"""Seeded synthetic inputs for the particle <-> dual-grid coupling step.

This module draws particles and fine-grid fluid fields; it holds none of the
coupling arithmetic (no binning, deposition, averaging, drag or projection).
Both the CUDA path (through its Python binding) and the FP64 oracle consume
what it returns, so neither side generates inputs for the other.

Random numbers come from numpy's Philox-4x32-10 counter-based generator
(Salmon et al., SC'11), one generator per (workload, seed).

The paper (Sec. 3) runs its benchmarks on an experimental dam-break and a
10M-particle layered bed whose case files are not available.  The workloads
below are synthetic stand-ins with the shapes, sizes and value distributions
named for this library's benchmarks:

* ``tiny``           unit cube, fine 32^3, ratio 4, 10,000 spheres, Taylor-Green fluid, FP64.
* ``packed_bed``     1x1x2 box, fine 256x256x512, ratio 4, 4M spheres in a jittered
                     lattice, 64 per packed bulk cell (porosity ~0.44), upward inflow, FP32.
* ``clustered_bed``  1x1x0.5 box, fine 512x512x256, ratio 4, 32M log-normal spheres in
                     200 Gaussian clusters, upward inflow, gravity, FP32.

Fluid properties everywhere are those of the paper's dam-break liquid and
particles (Sec. 3.2): rho_f = 1000, mu_f = 1e-3, rho_p = 2500.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

RHO_F = 1000.0
MU_F = 1.0e-3
RHO_P = 2500.0

DRAG_DI_FELICE = 0
DRAG_ERGUN_WEN_YU = 1
INTERP_TRILINEAR = 0
INTERP_CELL = 1


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    """Philox-4x32-10 generator keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[int(seed), int(stream)]))


def make_desc(origin, extent, fine_n, ratio, *, fp64: bool, law: int,
              eps_switch: float = 0.8, eps_min: float = 0.1,
              interp: int = INTERP_TRILINEAR, gravity=(0.0, 0.0, 0.0),
              rho_f: float = RHO_F, mu_f: float = MU_F, rho_p: float = RHO_P) -> dict:
    """Plain description of a coupling problem (mirrors ``cg_grid_desc``)."""
    return dict(origin=tuple(float(v) for v in origin),
                extent=tuple(float(v) for v in extent),
                fine_n=tuple(int(v) for v in fine_n),
                ratio=int(ratio), fp64=bool(fp64), law=int(law),
                eps_switch=float(eps_switch), eps_min=float(eps_min),
                interp=int(interp), gravity=tuple(float(v) for v in gravity),
                rho_f=float(rho_f), mu_f=float(mu_f), rho_p=float(rho_p))


@dataclass
class Workload:
    """One coupling instance: grids, particles and the fine fluid field.

    pos_d   (N, 4)  x, y, z, diameter     (dtype of the path)
    vel     (N, 4)  u, v, w, 0            (dtype of the path)
    u_fine  (3, nz, ny, nx) fine-cell-centre fluid velocity, x fastest
    """
    name: str
    desc: dict
    pos_d: np.ndarray
    vel: np.ndarray
    u_fine: np.ndarray
    dt: float = 0.0
    steps: int = 1
    notes: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos_d.shape[0])

    @property
    def dtype(self):
        return self.pos_d.dtype


def fine_centres(origin, extent, fine_n):
    """Fine-cell-centre coordinates per axis (x0 + (i + 1/2) h)."""
    return [origin[a] + (np.arange(fine_n[a], dtype=np.float64) + 0.5) * (extent[a] / fine_n[a])
            for a in range(3)]


def _pack(xyz, d, dtype):
    out = np.empty((xyz.shape[0], 4), dtype=dtype)
    out[:, :3] = xyz
    out[:, 3] = d
    return out


def tiny(seed: int = 0, n: int = 10_000, fine: int = 32, ratio: int = 4,
         d: float = 0.01, fp64: bool = True) -> Workload:
    """Unit cube, fine ``fine``^3, uniform positions, N(0, 0.05) velocities,
    u_f = 0.1 (sin x cos y cos z, -cos x sin y cos z, 0) at fine centres,
    Di Felice drag."""
    dtype = np.float64 if fp64 else np.float32
    rng = rng_for(seed, 1)
    desc = make_desc((0, 0, 0), (1, 1, 1), (fine,) * 3, ratio, fp64=fp64,
                     law=DRAG_DI_FELICE)
    xyz = rng.random((n, 3))
    vel3 = rng.normal(0.0, 0.05, (n, 3))
    cx, cy, cz = fine_centres(desc["origin"], desc["extent"], desc["fine_n"])
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    u = np.empty((3,) + X.shape, dtype=dtype)
    u[0] = 0.1 * np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -0.1 * np.cos(X) * np.sin(Y) * np.cos(Z)
    u[2] = 0.0
    return Workload("tiny", desc, _pack(xyz, d, dtype), _pack(vel3, 0.0, dtype), u)


def packed_bed(seed: int = 0, fine_n=(256, 256, 512), ratio: int = 4,
               n: int = 4_000_000, d: float = 0.004, sites_per_cell: int = 4,
               jitter: float = 0.75, fp64: bool = False) -> Workload:
    """Domain 1 x 1 x 2.  Spheres on a lattice commensurate with the bulk
    grid (``sites_per_cell`` sites per bulk cell per axis, so 64 per packed
    cell and solid fraction 64 V_p / V_B = 0.562, porosity ~0.44), filled
    layer by layer from z = 0 (the last layer partial).  Each position is
    jittered by U(+-jitter * spacing) per axis, so particles near a cell
    face cross into the neighbour and counts vary from cell to cell.  Zero
    particle velocity.  Fluid u_f = (0, 0, 0.5) + N(0, 0.02) per component
    per fine cell.  Ergun / Wen-Yu drag switched at porosity 0.8.
    Particles are stored in lattice order (x fastest, then y, then layer)."""
    dtype = np.float64 if fp64 else np.float32
    rng = rng_for(seed, 2)
    extent = (1.0, 1.0, 2.0)
    desc = make_desc((0, 0, 0), extent, fine_n, ratio, fp64=fp64,
                     law=DRAG_ERGUN_WEN_YU, eps_switch=0.8)
    nb = [fine_n[a] // ratio for a in range(3)]
    sp = [extent[a] / nb[a] / sites_per_cell for a in range(3)]
    nlx, nly = nb[0] * sites_per_cell, nb[1] * sites_per_cell
    idx = np.arange(n, dtype=np.int64)
    i = idx % nlx
    j = (idx // nlx) % nly
    k = idx // (nlx * nly)
    xyz = np.empty((n, 3), dtype=np.float64)
    xyz[:, 0] = (i + 0.5) * sp[0]
    xyz[:, 1] = (j + 0.5) * sp[1]
    xyz[:, 2] = (k + 0.5) * sp[2]
    jit = rng.uniform(-jitter, jitter, (n, 3))
    for a in range(3):
        xyz[:, a] += jit[:, a] * sp[a]
    np.clip(xyz, 0.0, np.asarray(extent), out=xyz)
    vel = np.zeros((n, 4), dtype=dtype)
    nz, ny, nx = fine_n[2], fine_n[1], fine_n[0]
    u = rng.standard_normal((3, nz, ny, nx), dtype=np.float32 if not fp64 else np.float64)
    u *= dtype(0.02)
    u[2] += dtype(0.5)
    layers = int(math.ceil(n / (nlx * nly)))
    return Workload("packed_bed", desc, _pack(xyz, d, dtype), vel, u.astype(dtype, copy=False),
                    notes=dict(lattice_spacing=tuple(sp), layers=layers,
                               bed_height=layers * sp[2],
                               order="lattice order, layer by layer (close to cell order)"))


def clustered_bed(seed: int = 0, fine_n=(512, 512, 256), ratio: int = 4,
                  n: int = 32_000_000, n_clusters: int = 200, sigma: float = 0.05,
                  d_median: float = 0.002, d_sigma: float = 0.3, dt: float = 1.0e-4,
                  steps: int = 100, fp64: bool = False) -> Workload:
    """Domain 1 x 1 x 0.5 (cubic cells).  Log-normal diameters (median
    ``d_median``, log-sigma ``d_sigma``); ``n_clusters`` centres uniform in
    the domain; each particle joins a uniformly drawn cluster and is offset
    by N(0, sigma) per axis, redrawn until inside the domain.  Zero particle
    velocity, u_f as in ``packed_bed``, Di Felice drag, gravity (0, 0, -9.81),
    explicit Euler with ``dt``."""
    dtype = np.float64 if fp64 else np.float32
    rng = rng_for(seed, 3)
    extent = (1.0, 1.0, 0.5)
    desc = make_desc((0, 0, 0), extent, fine_n, ratio, fp64=fp64,
                     law=DRAG_DI_FELICE, gravity=(0.0, 0.0, -9.81))
    L = np.asarray(extent)
    centres = rng.random((n_clusters, 3)) * L
    member = rng.integers(0, n_clusters, n)
    xyz = centres[member] + rng.normal(0.0, sigma, (n, 3))
    bad = np.nonzero(((xyz < 0.0) | (xyz > L)).any(axis=1))[0]
    while bad.size:
        xyz[bad] = centres[member[bad]] + rng.normal(0.0, sigma, (bad.size, 3))
        sub = ((xyz[bad] < 0.0) | (xyz[bad] > L)).any(axis=1)
        bad = bad[sub]
    dd = d_median * np.exp(d_sigma * rng.standard_normal(n))
    vel = np.zeros((n, 4), dtype=dtype)
    nz, ny, nx = fine_n[2], fine_n[1], fine_n[0]
    u = rng.standard_normal((3, nz, ny, nx), dtype=np.float32 if not fp64 else np.float64)
    u *= dtype(0.02)
    u[2] += dtype(0.5)
    pos = _pack(xyz, dd, dtype)
    # positions exactly at the upper face after rounding to the path dtype stay inside
    return Workload("clustered_bed", desc, pos, vel, u.astype(dtype, copy=False),
                    dt=dt, steps=steps,
                    notes=dict(order="draw order: each particle in a uniformly drawn cluster "
                                     "(no spatial order)"))


def medium_clustered_bed(seed: int = 0, fp64: bool = False) -> Workload:
    """Clustered bed at 1/8 scale: fine 256x256x128, ratio 4, 4,000,000
    spheres, 200 clusters (same particles per bulk cell as the full bed)."""
    return clustered_bed(seed, fine_n=(256, 256, 128), ratio=4, n=4_000_000, fp64=fp64)


def small_packed_bed(seed: int = 0, fp64: bool = False) -> Workload:
    """Packed bed at 1/64 of the volume count: fine 64x64x128, ratio 4,
    62,500 spheres of d = 0.016 (same porosity ~0.4, same bed height)."""
    return packed_bed(seed, fine_n=(64, 64, 128), ratio=4, n=62_500, d=0.016,
                      fp64=fp64)


def small_clustered_bed(seed: int = 0, fp64: bool = False) -> Workload:
    """Clustered bed at 1/64 scale: fine 128x128x64, ratio 4, 500,000
    spheres, 200 clusters."""
    return clustered_bed(seed, fine_n=(128, 128, 64), ratio=4, n=500_000, fp64=fp64)


def batch_instance(seed: int, k: int, edge: int, ratio: int, n: int, d: float) -> Workload:
    """Instance k of a batch: unit cube, fine edge^3, the given ratio, n
    spheres of diameter d uniform in the domain, N(0, 0.05) velocities,
    the Taylor-Green field of ``tiny``, Di Felice drag, FP32."""
    rng = rng_for(seed, 100 + k)
    desc = make_desc((0, 0, 0), (1, 1, 1), (edge,) * 3, ratio, fp64=False, law=DRAG_DI_FELICE)
    xyz = rng.random((n, 3))
    vel3 = rng.normal(0.0, 0.05, (n, 3))
    cx, cy, cz = fine_centres(desc["origin"], desc["extent"], desc["fine_n"])
    u = np.empty((3, edge, edge, edge), dtype=np.float32)
    u[0] = (0.1 * np.sin(cx)[None, None, :] * np.cos(cy)[None, :, None] * np.cos(cz)[:, None, None])
    u[1] = (-0.1 * np.cos(cx)[None, None, :] * np.sin(cy)[None, :, None] * np.cos(cz)[:, None, None])
    u[2] = 0.0
    return Workload(f"batch_{k}", desc, _pack(xyz, d, np.float32), _pack(vel3, 0.0, np.float32), u)


def uneven_batch(seed: int = 0, count: int = 64, edges=(32, 64, 96, 128), ratios=(2, 4, 8),
                 n_range=(10_000, 2_000_000), d_range=(0.002, 0.01)) -> list:
    """Independent instances of uneven sizes: per instance a fine edge from
    ``edges``, a ratio from ``ratios``, a particle count log-uniform in
    ``n_range`` and a diameter uniform in ``d_range`` (all from the seed)."""
    rng = rng_for(seed, 99)
    out = []
    for k in range(count):
        edge = int(rng.choice(edges))
        ratio = int(rng.choice(ratios))
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        d = float(rng.uniform(*d_range))
        out.append(batch_instance(seed, k, edge, ratio, n, d))
    return out


def evolved_field(w: Workload, seed: int = 0, amp: float = 0.05) -> np.ndarray:
    """A later fine velocity field for the stale / fresh closure cases:
    the workload's field plus a smooth large-scale swirl of amplitude
    ``amp`` and white noise of amplitude ``amp / 4`` per fine cell."""
    rng = rng_for(seed, 9)
    d = w.desc
    cx, cy, cz = fine_centres(d["origin"], d["extent"], d["fine_n"])
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    kx, ky, kz = (2 * np.pi / d["extent"][a] for a in range(3))
    u = w.u_fine.astype(np.float64, copy=True)
    u[0] += amp * np.sin(ky * Y) * np.cos(kz * Z)
    u[1] += amp * np.sin(kz * Z) * np.cos(kx * X)
    u[2] += amp * np.sin(kx * X) * np.cos(ky * Y)
    u += (amp / 4) * rng.normal(size=u.shape)
    return u.astype(w.dtype)


WORKLOADS = {
    "tiny": tiny,
    "packed_bed": packed_bed,
    "clustered_bed": clustered_bed,
    "small_packed_bed": small_packed_bed,
    "small_clustered_bed": small_clustered_bed,
    "medium_clustered_bed": medium_clustered_bed,
}
