"""Synthetic workloads: specimen recipes, material parameters and boundary conditions.

Units throughout: mm, N, MPa, tonne, s (so density is in t/mm^3 and velocity in mm/s).

The paper's own specimens (its data-availability archive) are not available, so each workload is a
seeded synthetic cube that stands in for one of the paper's benchmark families (Sec. 4):
  * elastic_vibration  -- free elastic vibration (Sec. 4.1), 25 mm cube, ~18k facets, FP64;
  * uniaxial_tension   -- tensile fracture to softening (dog-bone test, Sec. 4.3), 50 mm cube,
                          ~1.8M facets, FP32 facets / FP64 particle state;
  * confined_compression -- hydrostatic + triaxial compression with strain hardening (uniaxial-strain
                          test, Sec. 4.2), 100 mm cube, ~12.5M facets, mixed precision;
  * batched_unconfined_compression -- 64 random cubes of edge U(30, 60) mm, d = 2..4 mm, unconfined
                          compression between frictionless ("free") platens (Sec. 4.5), stepped as one
                          batch; particle counts scale with volume from uniaxial_tension's density;
  * adjoint_uniaxial_tension -- the uniaxial_tension cube pulled slowly (top u_z at 5 mm/s): 5000 steps
                          stay elastic and before the peak; gradient of the mean top reaction with
                          respect to every facet's E0, alpha, sigma_t (the paper has no derivatives).

Boundary-condition codes per degree of freedom (u_x, u_y, u_z, theta_x, theta_y, theta_z):
  0 = free, 1 = fixed (velocity 0), 2 = prescribed velocity bc_vel * ramp(t),
  ramp(t) = clamp(t / ramp_time, 0, 1) (ramp(t) = 1 when ramp_time <= 0).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .specimen import Specimen, make_cube_specimen

FREE, FIXED, PRESCRIBED = 0, 1, 2

# Paper, Appendix A, Table of material parameters (converted to mm-N-MPa-t-s).
TABLE_A = dict(
    rho=2380e-12,      # 2380 kg/m^3
    E0=60273.0,        # MPa
    alpha=0.25,
    sigma_t=3.44,      # MPa
    l_t=500.0,         # mm
    r_st=2.6,          # sigma_s / sigma_t
    n_t=0.4,
    sigma_c0=150.0,    # MPa
    Hc0_E0=0.40,
    Hc1_E0=0.1,
    kc0=4.0,
    kc1=1.0,
    kc2=5.0,
    kc3=0.1,
    mu0=0.4,
    mu_inf=0.0,
    sigma_N0=600.0,    # MPa
    Ed_E0=1.0,
    beta=0.0,
    k_t=0.0,
    r_s=0.0,
    elastic=0,
)

# Parameters the synthetic workloads use: the values the workload definitions name, Table A for the
# rest (density 2400 kg/m^3, E0 = 43.7 GPa, alpha = 0.29, sigma_t = 4.03 MPa, l_t = 120 mm,
# sigma_s/sigma_t = 2.7, n_t = 0.2, kappa_c0 = 2, mu_0 = 0.2).
WORKLOAD_MATERIAL = dict(TABLE_A, rho=2400e-12, E0=43700.0, alpha=0.29, sigma_t=4.03, l_t=120.0,
                         r_st=2.7, n_t=0.2, kc0=2.0, mu0=0.2)

MATERIAL_FIELDS = ("rho", "E0", "alpha", "sigma_t", "l_t", "r_st", "n_t", "sigma_c0", "Hc0_E0", "Hc1_E0",
                   "kc0", "kc1", "kc2", "kc3", "mu0", "mu_inf", "sigma_N0", "Ed_E0", "beta", "k_t", "r_s")


@dataclasses.dataclass
class BoundaryConditions:
    mask: np.ndarray        # (N, 6) int32
    vel: np.ndarray         # (N, 6) float64, mm/s (rad/s for rotations)
    ramp_time: float        # s
    v0: np.ndarray          # (N, 6) float64 initial velocity


@dataclasses.dataclass
class Workload:
    name: str
    edge: float
    d_min: float
    d_max: float
    n_particles: int
    seed: int
    material: dict
    precision: str          # "fp64" or "mixed"
    steps: int
    dt_factor: float = 0.9
    # Fixed time step of the benchmark runs (s): 0.9 of the critical step 2 / sqrt(lambda_max(M^-1 K))
    # of the seeded specimen (the oracle's power iteration: 2.31e-7 s for the 50 mm cubes, 2.52e-7 s
    # for the 100 mm cube, 4.60e-7 s for the 25 mm cube), rounded down, so that every arm of a
    # comparison steps with the same dt.  0 = estimate per run.
    dt: float = 0.0
    # Untimed steps of the loading history before a benchmark's warm-up and timed window: enough for
    # the loading wave (~1 mm per step) to cross the specimen, so that the timed steps see every facet
    # strained rather than the law's zero-strain path.
    preroll: int = 200

    def specimen(self) -> Specimen:
        return make_cube_specimen(self.edge, self.d_min, self.d_max, self.n_particles, self.seed)


def free_bc(n: int) -> BoundaryConditions:
    return BoundaryConditions(mask=np.zeros((n, 6), np.int32), vel=np.zeros((n, 6)), ramp_time=0.0,
                              v0=np.zeros((n, 6)))


def elastic_vibration_bc(spec: Specimen, amplitude: float = 10.0) -> BoundaryConditions:
    """Bottom face fixed in all six DOFs; initial velocity v_x = A sin(pi z / (2 L)) (mm/s)."""
    bc = free_bc(spec.n_particles)
    bot = spec.face_nodes(2, 0)
    bc.mask[bot, :] = FIXED
    bc.v0[:, 0] = amplitude * np.sin(np.pi * spec.x[:, 2] / (2.0 * spec.edge))
    bc.v0[bot, :] = 0.0
    return bc


def uniaxial_tension_bc(spec: Specimen, velocity: float = 50.0, ramp_time: float = 4e-4) -> BoundaryConditions:
    """Tension as in the paper's dog-bone test (Sec. 4.3), on a cube.

    Bottom face: u_x, u_y, u_z, theta_x, theta_y fixed.  Top face: the same, except u_z moves at
    +velocity (ramped linearly over ramp_time).  theta_z is free on both faces.
    """
    bc = free_bc(spec.n_particles)
    bot, top = spec.face_nodes(2, 0), spec.face_nodes(2, 1)
    for nodes in (bot, top):
        bc.mask[np.ix_(nodes, [0, 1, 2, 3, 4])] = FIXED
    bc.mask[top, 2] = PRESCRIBED
    bc.vel[top, 2] = velocity
    bc.ramp_time = ramp_time
    return bc


def confined_compression_bc(spec: Specimen, velocity: float = 25.0, phase: int = 1,
                            ramp_time: float = 2e-4) -> BoundaryConditions:
    """Hydrostatic (phase 1) then triaxial (phase 2) compression of a cube.

    Phase 1: the normal displacement of every face moves inward at `velocity`.  Phase 2: the four
    lateral faces hold their normal displacement (fixed) while top and bottom keep moving inward.
    Tangential translations and rotations of face nodes stay free.
    """
    bc = free_bc(spec.n_particles)
    for ax in range(3):
        for side, sgn in ((0, 1.0), (1, -1.0)):
            nodes = spec.face_nodes(ax, side)
            if phase == 2 and ax < 2:
                bc.mask[nodes, ax] = FIXED
                bc.vel[nodes, ax] = 0.0
            else:
                bc.mask[nodes, ax] = PRESCRIBED
                bc.vel[nodes, ax] = sgn * velocity
    bc.ramp_time = ramp_time
    return bc


def adjoint_tension_bc(spec: Specimen, velocity: float = 5.0, ramp_time: float = 4e-4) -> BoundaryConditions:
    """uniaxial_tension_bc at a slow rate: 5000 steps end at about 60 % of the peak load."""
    return uniaxial_tension_bc(spec, velocity=velocity, ramp_time=ramp_time)


def unconfined_compression_bc(spec: Specimen, velocity: float = 50.0, ramp_time: float = 2e-4) -> BoundaryConditions:
    """Unconfined compression with free platens as in Sec. 4.5: on the top and bottom faces u_z is
    prescribed (top moving down at `velocity`, bottom held) and theta_x, theta_y are fixed, while u_x,
    u_y and theta_z stay free; the node nearest each platen centre also holds u_x, u_y, theta_z."""
    bc = free_bc(spec.n_particles)
    bot, top = spec.face_nodes(2, 0), spec.face_nodes(2, 1)
    for nodes in (bot, top):
        bc.mask[np.ix_(nodes, [3, 4])] = FIXED
        c = nodes[np.argmin(np.linalg.norm(spec.x[nodes, :2] - 0.5 * spec.edge, axis=1))]
        bc.mask[c, [0, 1, 5]] = FIXED
    bc.mask[bot, 2] = FIXED
    bc.mask[top, 2] = PRESCRIBED
    bc.vel[top, 2] = -velocity
    bc.ramp_time = ramp_time
    return bc


# Batched workload: n cubes, edges uniform in [30, 60] mm (seeded), particle count at the density of
# uniaxial_tension (25000 particles in a 50 mm cube).
BATCH_DENSITY = 25000.0 / 50.0 ** 3


def batch_recipe(n: int = 64, seed: int = 1):
    rng = np.random.default_rng(seed)
    edges = rng.uniform(30.0, 60.0, n)
    return [(float(L), 2.0, 4.0, int(round(BATCH_DENSITY * L ** 3)), seed * 1000 + i) for i, L in enumerate(edges)]


def _make(args):
    L, dmin, dmax, n, sd = args
    return make_cube_specimen(L, dmin, dmax, n, sd)


def batch_specimens(n: int = 64, seed: int = 1, processes: int | None = None):
    """Generate the batch in parallel worker processes (spawned, so no CUDA context is inherited)."""
    import multiprocessing as mp
    import os as _os

    recipe = batch_recipe(n, seed)
    procs = processes or max(1, min(len(recipe), (_os.cpu_count() or 2)))
    if procs == 1:
        return [_make(r) for r in recipe]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_make, recipe)


WORKLOADS = {
    "elastic_vibration": Workload("elastic_vibration", 25.0, 4.0, 8.0, 420, 1, dict(WORKLOAD_MATERIAL, elastic=1),
                                  "fp64", 2000, dt=4.1e-7, preroll=0),
    "uniaxial_tension": Workload("uniaxial_tension", 50.0, 2.0, 4.0, 25000, 1, dict(WORKLOAD_MATERIAL), "mixed",
                                 200000, dt=2.0e-7, preroll=200),
    "confined_compression": Workload("confined_compression", 100.0, 3.0, 6.0, 165000, 1,
                                     dict(WORKLOAD_MATERIAL), "mixed", 50000, dt=2.2e-7, preroll=100),
    "adjoint_uniaxial_tension": Workload("adjoint_uniaxial_tension", 50.0, 2.0, 4.0, 25000, 1,
                                         dict(WORKLOAD_MATERIAL), "mixed", 5000, dt=2.0e-7, preroll=0),
}
# (the batched workload is built by batch_specimens / batch_recipe; material WORKLOAD_MATERIAL with
# the friction of the workload definition: mu_0 = 0.2, mu_inf = 0, sigma_N0 = 600 MPa)


def workload_bc(name: str, spec: Specimen) -> BoundaryConditions:
    if name == "elastic_vibration":
        return elastic_vibration_bc(spec)
    if name == "uniaxial_tension":
        return uniaxial_tension_bc(spec)
    if name == "confined_compression":
        return confined_compression_bc(spec)
    if name == "batched_unconfined_compression":
        return unconfined_compression_bc(spec)
    if name == "adjoint_uniaxial_tension":
        return adjoint_tension_bc(spec)
    raise KeyError(name)
