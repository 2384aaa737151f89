"""Seeded synthetic inputs for the fiber-diffraction hot path.

This module only draws and packages inputs: atoms, synthetic form-factor
coefficients, cells, broadening parameters and detector geometry.  It holds
none of the method's arithmetic (no reciprocal basis, no structure factors,
no profiles, no Ewald map), so both the FP64 oracle tests and the GPU path can
consume the same inputs without sharing any of the computation.

The five workloads follow the hot-path scope of the paper (structure factors
by direct summation, Eq. structure_factor; shell quadrature, Eqs. gnomonic and
node_weight; Hosemann disorder, Eqs. Z, Neff, Ipara; Lorentz-corrected Ewald
projection, Eq. lorentz and Sect. "Analytical Solution of the Ewald
Diffraction Condition").  The paper's own structures (cellulose, chitin, CTA,
DNA) are not available, so seeded synthetic atoms stand in for them.

Random stream: ``numpy.random.Generator(PCG64(2608232450 + config_id))``;
model ``m`` of the batched workload uses seed ``(2608232450 + 4) * 1000 + m``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List

import numpy as np

SEED_BASE = 2608232450
ELEMENTS = ("C", "N", "O", "S")
ELEMENT_P = (0.5, 0.2, 0.25, 0.05)

LINESHAPE_SINC = 0
LINESHAPE_HOSEMANN = 1
LINESHAPE_GAUSS = 2
INTENSITY_NONE = 0
INTENSITY_HOSEMANN = 1


@dataclass
class Atoms:
    frac: np.ndarray          # [n, 3] float64 fractional coordinates
    B: np.ndarray             # [n] float64 isotropic B (A^2)
    occ: np.ndarray           # [n] float64 occupancy (1 everywhere, as in the paper)
    elem: np.ndarray          # [n] uint8 element index
    ff: np.ndarray            # [n_elem, 9] float64: a1..a4, b1..b4, c

    @property
    def n(self) -> int:
        return int(self.frac.shape[0])


@dataclass
class Broadening:
    L: tuple                  # crystallite size along a, b, c (A)
    g: tuple                  # Hosemann g along a, b, c
    B_axis: tuple = (0.0, 0.0, 0.0)   # axis Debye-Waller B_a, B_b, B_c (A^2)
    lineshape: int = LINESHAPE_HOSEMANN
    intensity_model: int = INTENSITY_HOSEMANN
    sigma: float = 0.0        # Gaussian orientation width (rad)
    gamma: float = 0.0        # Lorentzian orientation HWHM (rad)
    sigma_r: float = 1e-4     # radial shell width (1/A)
    T: float = 0.0            # patch half-extent, tangent units
    n_nodes: int = 32         # shell nodes per axis
    K_z: float = 3.0          # sinc support, in zeros


@dataclass
class Geometry:
    wavelength: float         # A
    distance: float           # sample-detector distance (mm)
    pixel: float              # mm
    n_x: int
    n_y: int
    fiber_axis: tuple = (0.0, 0.0, 1.0)
    beam_axis: tuple = (1.0, 0.0, 0.0)
    delta_L: float = 1e-5     # Lorentz regulariser (1/A)


@dataclass
class Problem:
    name: str
    cell: tuple               # a, b, c (A), alpha, beta, gamma (rad)
    atoms: Atoms
    d_min: float
    d_max: float
    br: Broadening
    geom: Geometry
    seed: int = 0
    extra: dict = field(default_factory=dict)


def patch_extent(sigma: float, gamma: float) -> float:
    """Patch half-extent in tangent units, scaled by the combined width
    sqrt(sigma^2 + gamma^2) as the paper prescribes for heavy tails (Sect.
    "Angular peak shapes"): T = tan(3 sqrt(sigma^2 + gamma^2))."""
    return math.tan(3.0 * math.sqrt(sigma * sigma + gamma * gamma))


def distance_for_resolution(n_min_px: int, pixel: float, wavelength: float, d_min: float) -> float:
    """Detector distance rule of Eq. SF: SF = 0.9 * min(det) * p / (2 tan 2theta_max)."""
    two_theta = 2.0 * math.asin(wavelength / (2.0 * d_min))
    return 0.9 * n_min_px * pixel / (2.0 * math.tan(two_theta))


def _form_factors(rng: np.random.Generator, n_elem: int = 4) -> np.ndarray:
    ff = np.empty((n_elem, 9), dtype=np.float64)
    for e in range(n_elem):
        ff[e, 0:4] = rng.uniform(0.5, 3.0, size=4)
        ff[e, 4:8] = rng.uniform(0.5, 40.0, size=4)
        ff[e, 8] = rng.uniform(0.0, 1.0)
    return ff


def _elements(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.choice(len(ELEMENTS), size=n, p=np.asarray(ELEMENT_P)).astype(np.uint8)


def _uniform_atoms(rng: np.random.Generator, n: int) -> Atoms:
    ff = _form_factors(rng)
    elem = _elements(rng, n)
    frac = rng.uniform(0.0, 1.0, size=(n, 3))
    B = rng.uniform(10.0, 30.0, size=n)
    return Atoms(frac=frac, B=B, occ=np.ones(n), elem=elem, ff=ff)


def _hexagonal_frame(a: float, c: float) -> np.ndarray:
    """Cartesian edge vectors (rows) of the a=b, gamma=120 deg cell in the
    frame used to place the synthetic helix: c along z, b along y."""
    g = math.radians(120.0)
    return np.array([[a * math.sin(g), a * math.cos(g), 0.0],
                     [0.0, a, 0.0],
                     [0.0, 0.0, c]])


def _helix_atoms(rng: np.random.Generator, n_res: int, a: float, c: float,
                 radius=5.0, rise=1.5, twist_deg=100.0, jitter=0.3):
    """400 residues x 5 atoms on a helix (radius 5 A, rise 1.5 A, 100 deg per
    residue) about the cell's centre line, with seeded +-0.3 A offsets.
    Returns Cartesian positions (A) and the frame used to place them."""
    E = _hexagonal_frame(a, c)
    centre = 0.5 * E[0] + 0.5 * E[1]
    r = np.arange(n_res, dtype=np.float64)
    ang = np.radians(twist_deg) * r
    res = centre[None, :] + np.stack([radius * np.cos(ang), radius * np.sin(ang), rise * r], axis=1)
    xyz = np.repeat(res, 5, axis=0) + rng.uniform(-jitter, jitter, size=(5 * n_res, 3))
    return xyz, E


def _cart_to_frac_wrapped(xyz: np.ndarray, E: np.ndarray) -> np.ndarray:
    frac = np.linalg.solve(E.T, xyz.T).T
    return frac - np.floor(frac)


def config0() -> Problem:
    """Small plain case: 120 atoms, orthorhombic 9x9x15 A, d >= 2.5 A,
    Gaussian orientation 5 deg, sinc lineshape, 32x32 nodes, 256^2 detector."""
    seed = SEED_BASE + 0
    rng = np.random.Generator(np.random.PCG64(seed))
    atoms = _uniform_atoms(rng, 120)
    sig = math.radians(5.0)
    br = Broadening(L=(100.0, 100.0, 100.0), g=(0.0, 0.0, 0.0),
                    lineshape=LINESHAPE_SINC, intensity_model=INTENSITY_NONE,
                    sigma=sig, gamma=0.0, T=patch_extent(sig, 0.0), n_nodes=32)
    geom = Geometry(wavelength=1.0, distance=100.0, pixel=0.1, n_x=256, n_y=256)
    return Problem("c0_plain_small", (9.0, 9.0, 15.0, math.pi / 2, math.pi / 2, math.pi / 2),
                   atoms, 2.5, 0.0, br, geom, seed)


def config1() -> Problem:
    """Helical fiber model: 2,000 atoms on a helix in a hexagonal 20x20x28 A
    cell, d >= 2.0 A, Voigt orientation (3 deg, 2 deg), size 200x200x300 A,
    Hosemann g = 2 % along a and b, 64x64 nodes, 1024^2 detector."""
    seed = SEED_BASE + 1
    rng = np.random.Generator(np.random.PCG64(seed))
    ff = _form_factors(rng)
    elem = _elements(rng, 2000)
    B = rng.uniform(10.0, 30.0, size=2000)
    xyz, E = _helix_atoms(rng, 400, 20.0, 28.0)
    frac = _cart_to_frac_wrapped(xyz, E)
    atoms = Atoms(frac=frac, B=B, occ=np.ones(2000), elem=elem, ff=ff)
    sig, gam = math.radians(3.0), math.radians(2.0)
    br = Broadening(L=(200.0, 200.0, 300.0), g=(0.02, 0.02, 0.0),
                    lineshape=LINESHAPE_HOSEMANN, intensity_model=INTENSITY_HOSEMANN,
                    sigma=sig, gamma=gam, T=patch_extent(sig, gam), n_nodes=64)
    geom = Geometry(wavelength=1.0, distance=150.0, pixel=0.1, n_x=1024, n_y=1024)
    p = Problem("c1_helix_fp32", (20.0, 20.0, 28.0, math.pi / 2, math.pi / 2, math.radians(120.0)),
                atoms, 2.0, 0.0, br, geom, seed)
    p.extra["cart"] = xyz
    p.extra["frame"] = E
    return p


def config2(g: float = 0.01) -> Problem:
    """Large forward: 20,000 uniform atoms in a 50x50x70 A cell, d >= 1.5 A,
    Lorentzian orientation 4 deg, size 300 A, Hosemann g (1 % or 4 %),
    128x128 nodes, 2048^2 detector with 0.075 mm pixels at 200 mm."""
    seed = SEED_BASE + 2
    rng = np.random.Generator(np.random.PCG64(seed))
    atoms = _uniform_atoms(rng, 20000)
    gam = math.radians(4.0)
    br = Broadening(L=(300.0, 300.0, 300.0), g=(g, g, g),
                    lineshape=LINESHAPE_HOSEMANN, intensity_model=INTENSITY_HOSEMANN,
                    sigma=0.0, gamma=gam, T=patch_extent(0.0, gam), n_nodes=128)
    geom = Geometry(wavelength=1.0, distance=200.0, pixel=0.075, n_x=2048, n_y=2048)
    return Problem("c2_large_g%02d" % int(round(g * 100)),
                   (50.0, 50.0, 70.0, math.pi / 2, math.pi / 2, math.pi / 2),
                   atoms, 1.5, 0.0, br, geom, seed)


def config3():
    """Refinement on the helical system: returns (model, target) where the
    target's parameters are seeded perturbations of the model's: Cartesian
    coordinates +-0.2 A, B +-5 A^2, all sizes x (1 +- 20 %), sigma +-1 deg,
    g_a = g_b +- 1 %; gamma unchanged."""
    model = config1()
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 3))
    xyz = model.extra["cart"] + rng.uniform(-0.2, 0.2, size=model.extra["cart"].shape)
    B = model.atoms.B + rng.uniform(-5.0, 5.0, size=model.atoms.n)
    fL = 1.0 + rng.uniform(-0.2, 0.2)
    dsig = math.radians(rng.uniform(-1.0, 1.0))
    dg = rng.uniform(-0.01, 0.01)
    frac = _cart_to_frac_wrapped(xyz, model.extra["frame"])
    atoms = replace(model.atoms, frac=frac, B=B)
    br = replace(model.br, L=tuple(fL * x for x in model.br.L),
                 sigma=model.br.sigma + dsig,
                 g=(model.br.g[0] + dg, model.br.g[1] + dg, model.br.g[2]))
    target = replace(model, name="c3_target", atoms=atoms, br=br, seed=SEED_BASE + 3)
    target.extra = {"cart": xyz, "frame": model.extra["frame"]}
    return model, target


def config4_model(m: int) -> Problem:
    """Model m of the batched-refinement workload: log-uniform 500-8,000 atoms,
    orthorhombic edges U[10, 40] A, d >= 2.0 A, ROI side 16*round(U[16, 64]) px
    (0.1 mm pixels, distance by Eq. SF), Gaussian sigma~U[2,6] deg or Voigt
    (sigma, gamma)~U[1,4] deg each with p = 1/2, g~U[0, 5 %], L~U[100, 300] A,
    64x64 nodes."""
    seed = (SEED_BASE + 4) * 1000 + m
    rng = np.random.Generator(np.random.PCG64(seed))
    n_atoms = int(round(math.exp(rng.uniform(math.log(500.0), math.log(8000.0)))))
    edges = rng.uniform(10.0, 40.0, size=3)
    side = 16 * int(round(rng.uniform(16.0, 64.0)))
    if rng.uniform() < 0.5:
        sig, gam = math.radians(rng.uniform(2.0, 6.0)), 0.0
    else:
        sig, gam = math.radians(rng.uniform(1.0, 4.0)), math.radians(rng.uniform(1.0, 4.0))
    g = float(rng.uniform(0.0, 0.05))
    L = float(rng.uniform(100.0, 300.0))
    atoms = _uniform_atoms(rng, n_atoms)
    br = Broadening(L=(L, L, L), g=(g, g, g), lineshape=LINESHAPE_HOSEMANN,
                    intensity_model=INTENSITY_HOSEMANN, sigma=sig, gamma=gam,
                    T=patch_extent(sig, gam), n_nodes=64)
    geom = Geometry(wavelength=1.0, distance=distance_for_resolution(side, 0.1, 1.0, 2.0),
                    pixel=0.1, n_x=side, n_y=side)
    return Problem("c4_model%03d" % m, (float(edges[0]), float(edges[1]), float(edges[2]),
                                        math.pi / 2, math.pi / 2, math.pi / 2),
                   atoms, 2.0, 0.0, br, geom, seed)


def config4(n_models: int = 256) -> List[Problem]:
    return [config4_model(m) for m in range(n_models)]


def config4_target(model: Problem, m: int) -> Problem:
    """Seeded perturbation of batched model m (as for the helix refinement):
    Cartesian coordinates +-0.2 A (orthorhombic cell: fractional +-0.2/edge),
    B +-5 A^2, sizes x (1 +- 20 %), sigma +-1 deg (gamma unchanged), g +-1 %
    (kept >= 0)."""
    rng = np.random.Generator(np.random.PCG64((SEED_BASE + 4) * 1000 + 500 + m))
    edges = np.array(model.cell[:3])
    frac = model.atoms.frac + rng.uniform(-0.2, 0.2, size=model.atoms.frac.shape) / edges[None, :]
    B = model.atoms.B + rng.uniform(-5.0, 5.0, size=model.atoms.n)
    fL = 1.0 + rng.uniform(-0.2, 0.2)
    dsig = math.radians(rng.uniform(-1.0, 1.0))
    dg = rng.uniform(-0.01, 0.01)
    br = replace(model.br, L=tuple(fL * x for x in model.br.L), sigma=max(model.br.sigma + dsig, math.radians(0.5)),
                 g=tuple(max(0.0, x + dg) for x in model.br.g))
    return replace(model, name=model.name + "_target", atoms=replace(model.atoms, frac=frac, B=B), br=br)


def small_batch(n_models: int = 5) -> List[Problem]:
    """Reduced batched-refinement models for tests: the config-4 recipe with
    the detector cut to a seeded 40-72 px ROI of the same angular coverage and
    at most 600 atoms."""
    out = []
    for m in range(n_models):
        p = config4_model(m)
        rng = np.random.Generator(np.random.PCG64(SEED_BASE + 40 + m))
        side = int(rng.integers(40, 73))
        k = min(p.atoms.n, 600)
        atoms = Atoms(frac=p.atoms.frac[:k].copy(), B=p.atoms.B[:k].copy(), occ=p.atoms.occ[:k].copy(),
                      elem=p.atoms.elem[:k].copy(), ff=p.atoms.ff)
        geom = replace(p.geom, n_x=side, n_y=side + int(rng.integers(0, 9)), pixel=p.geom.pixel * p.geom.n_x / side)
        br = replace(p.br, n_nodes=20)
        out.append(replace(p, name="small_batch%d" % m, atoms=atoms, geom=geom, br=br, d_min=3.0))
    return out


# ---------------------------------------------------------------------------
# Reduced variants: same recipes, sized so the FP64 oracle finishes a whole
# detector in seconds.  Each spans several 16x8-pixel tiles and leaves ragged
# detector edges.
# ---------------------------------------------------------------------------

def small_sinc() -> Problem:
    """Config-0 recipe on a 72x60 detector with 0.35 mm pixels (same angular
    coverage as 256 x 0.1 mm) and 16x16 nodes."""
    p = config0()
    br = replace(p.br, n_nodes=16)
    geom = replace(p.geom, n_x=72, n_y=60, pixel=0.35)
    return replace(p, name="small_sinc", br=br, geom=geom)


def small_helix() -> Problem:
    """Config-1 recipe reduced: 60 residues (300 atoms), d >= 3.0 A, 24x24
    nodes, 90x70 detector with 0.9 mm pixels at 150 mm."""
    seed = SEED_BASE + 11
    rng = np.random.Generator(np.random.PCG64(seed))
    ff = _form_factors(rng)
    elem = _elements(rng, 300)
    B = rng.uniform(10.0, 30.0, size=300)
    xyz, E = _helix_atoms(rng, 60, 20.0, 28.0)
    atoms = Atoms(frac=_cart_to_frac_wrapped(xyz, E), B=B, occ=np.ones(300), elem=elem, ff=ff)
    sig, gam = math.radians(3.0), math.radians(2.0)
    br = Broadening(L=(200.0, 200.0, 300.0), g=(0.02, 0.02, 0.0),
                    lineshape=LINESHAPE_HOSEMANN, intensity_model=INTENSITY_HOSEMANN,
                    sigma=sig, gamma=gam, T=patch_extent(sig, gam), n_nodes=24)
    geom = Geometry(wavelength=1.0, distance=150.0, pixel=0.9, n_x=90, n_y=70)
    p = Problem("small_helix", (20.0, 20.0, 28.0, math.pi / 2, math.pi / 2, math.radians(120.0)),
                atoms, 3.0, 0.0, br, geom, seed)
    p.extra["cart"] = xyz
    p.extra["frame"] = E
    return p


def small_lorentz() -> Problem:
    """Config-2 recipe reduced: 400 atoms in the 50x50x70 A cell, d >= 4.5 A,
    Lorentzian 4 deg, g = 4 %, 20x20 nodes, 84x52 detector, 1.2 mm pixels."""
    seed = SEED_BASE + 12
    rng = np.random.Generator(np.random.PCG64(seed))
    atoms = _uniform_atoms(rng, 400)
    gam = math.radians(4.0)
    br = Broadening(L=(300.0, 300.0, 300.0), g=(0.04, 0.04, 0.04),
                    lineshape=LINESHAPE_HOSEMANN, intensity_model=INTENSITY_HOSEMANN,
                    sigma=0.0, gamma=gam, T=patch_extent(0.0, gam), n_nodes=20)
    geom = Geometry(wavelength=1.0, distance=200.0, pixel=1.2, n_x=84, n_y=52)
    return Problem("small_lorentz", (50.0, 50.0, 70.0, math.pi / 2, math.pi / 2, math.pi / 2),
                   atoms, 4.5, 0.0, br, geom, seed)


def small_gauss() -> Problem:
    """The reduced helix (small_helix) with the Gaussian lineshape of matched
    integral breadth instead of the Hosemann factor."""
    p = small_helix()
    return replace(p, name="small_gauss", br=replace(p.br, lineshape=LINESHAPE_GAUSS))


def tilted(p: Problem, tilt_deg: float) -> Problem:
    """The same problem with the fiber axis tilted by tilt_deg towards the
    beam (rotation about the detector's horizontal axis n x b)."""
    n = np.asarray(p.geom.fiber_axis, float)
    b = np.asarray(p.geom.beam_axis, float)
    n = n / np.linalg.norm(n)
    b = b / np.linalg.norm(b)
    t = math.radians(tilt_deg)
    nt = math.cos(t) * n - math.sin(t) * b
    return replace(p, name="%s_tilt%g" % (p.name, tilt_deg), geom=replace(p.geom, fiber_axis=tuple(float(x) for x in nt)))


def small_tilted() -> Problem:
    """The reduced helix with the fiber axis tilted by 20 deg towards the beam."""
    return tilted(small_helix(), 20.0)


def sample_brick(n_r: int, n_1: int, n_2: int):
    """Brick of 32 grid cells in which the scatter samples are ordered (a warp
    of the scatter kernel takes two consecutive bricks, one per query point of
    its lanes; consecutive bricks are neighbours along the last axis):
    4 x 4 x 2 (radial x angular x angular), the fastest shape measured, or
    2 x 4 x 4 when n_r is not a multiple of 4."""
    brick = (4, 4, 2) if n_r % 4 == 0 and n_2 % 2 == 0 else (2, 4, 4)
    if n_r % brick[0] or n_1 % brick[1] or n_2 % brick[2]:
        raise ValueError("grid must be a multiple of 4 x 4 x 2 or of 2 x 4 x 4")
    return brick


def scatter_samples(n_r: int, n_1: int, n_2: int, seed: int = SEED_BASE + 50) -> np.ndarray:
    """Seeded stratified samples for the scatter form: one jittered point in
    each cell of an n_r x n_1 x n_2 grid on [-1, 1]^3, float32 rows (x_r, x_1,
    x_2, q) with q = 8 / (n_r n_1 n_2), ordered in bricks of 32 cells (see
    `sample_brick`) so that every 32 consecutive samples are neighbours."""
    b_r, b_1, b_2 = sample_brick(n_r, n_1, n_2)
    rng = np.random.Generator(np.random.PCG64(seed))
    jit = rng.uniform(0.0, 1.0, size=(n_r, n_1, n_2, 3))
    out = np.empty((n_r * n_1 * n_2, 4), dtype=np.float32)
    k = 0
    for br in range(0, n_r, b_r):
        for b1 in range(0, n_1, b_1):
            for b2 in range(0, n_2, b_2):
                for ir in range(br, br + b_r):
                    for i1 in range(b1, b1 + b_1):
                        for i2 in range(b2, b2 + b_2):
                            j = jit[ir, i1, i2]
                            out[k] = (-1.0 + 2.0 * (ir + j[0]) / n_r, -1.0 + 2.0 * (i1 + j[1]) / n_1,
                                      -1.0 + 2.0 * (i2 + j[2]) / n_2, 8.0 / (n_r * n_1 * n_2))
                            k += 1
    return out


def scatter_samples_cauchy(n_r: int, n_1: int, n_2: int, scale: float, extent: float,
                           seed: int = SEED_BASE + 51) -> np.ndarray:
    """Seeded stratified samples for the scatter form whose angular coordinates
    are heavy-tailed: the paper samples the shell from a Cauchy distribution
    when the orientation distribution has a Lorentzian part, so that the slow
    tails are not cut off at the sampling stage (Sect. "Angular peak shapes").

    x_r is stratified uniform on [-1, 1].  x_1 and x_2 follow a Cauchy density
    of half-width `scale` (normalised units: tan(gamma) / T) truncated to
    |x| <= extent, drawn by inverse transform from stratified u:
    x = scale tan(theta), theta = theta_max (2u - 1), theta_max =
    atan(extent / scale), with density scale / ((scale^2 + x^2) 2 theta_max).
    extent > 1 reaches past the node patch by (extent - 1) T.  The weight
    q = 1 / (n pdf(x_r) pdf(x_1) pdf(x_2)) makes sum q f(x) an unbiased
    estimate of the integral of f over [-1, 1] x [-extent, extent]^2.  Rows
    (x_r, x_1, x_2, q) as float32, in bricks like scatter_samples."""
    b_r, b_1, b_2 = sample_brick(n_r, n_1, n_2)
    if not (scale > 0 and extent > 0):
        raise ValueError("scale and extent must be positive")
    rng = np.random.Generator(np.random.PCG64(seed))
    jit = rng.uniform(0.0, 1.0, size=(n_r, n_1, n_2, 3))
    th_max = math.atan(extent / scale)
    n = n_r * n_1 * n_2
    out = np.empty((n, 4), dtype=np.float32)
    k = 0
    for br in range(0, n_r, b_r):
        for b1 in range(0, n_1, b_1):
            for b2 in range(0, n_2, b_2):
                for ir in range(br, br + b_r):
                    for i1 in range(b1, b1 + b_1):
                        for i2 in range(b2, b2 + b_2):
                            j = jit[ir, i1, i2]
                            xr = -1.0 + 2.0 * (ir + j[0]) / n_r
                            th1 = th_max * (2.0 * (i1 + j[1]) / n_1 - 1.0)
                            th2 = th_max * (2.0 * (i2 + j[2]) / n_2 - 1.0)
                            x1, x2 = scale * math.tan(th1), scale * math.tan(th2)
                            pdf = (0.5 * scale / ((scale * scale + x1 * x1) * 2.0 * th_max)
                                   * scale / ((scale * scale + x2 * x2) * 2.0 * th_max))
                            out[k] = (xr, x1, x2, 1.0 / (n * pdf))
                            k += 1
    return out


def small_triclinic() -> Problem:
    """A general triclinic cell (alpha, beta, gamma != 90 deg), Voigt
    orientation, anisotropic g and axis B, 18x18 nodes, 64x48 detector;
    exercises every term the path has."""
    seed = SEED_BASE + 13
    rng = np.random.Generator(np.random.PCG64(seed))
    atoms = _uniform_atoms(rng, 60)
    sig, gam = math.radians(2.5), math.radians(1.5)
    br = Broadening(L=(120.0, 150.0, 90.0), g=(0.015, 0.03, 0.01), B_axis=(4.0, 8.0, 2.0),
                    lineshape=LINESHAPE_HOSEMANN, intensity_model=INTENSITY_HOSEMANN,
                    sigma=sig, gamma=gam, T=patch_extent(sig, gam), n_nodes=18)
    geom = Geometry(wavelength=1.0, distance=100.0, pixel=0.6, n_x=64, n_y=48)
    cell = (8.2, 10.4, 12.9, math.radians(80.37), math.radians(108.1), math.radians(95.4))
    return Problem("small_triclinic", cell, atoms, 3.2, 0.0, br, geom, seed)


# ---------------------------------------------------------------------------
# The paper's model figures with |F| = 1 (Figs. GvL and equator): a hexagonal
# cell a = b = 10 A, c = 5 A, gamma = 120 deg and a structure factor of one
# for every reflection.  Neither figure states its remaining parameters; the
# values below (d >= 2 A, crystallite size, detector) are this project's.
# ---------------------------------------------------------------------------

FIGURE_CELL = (10.0, 10.0, 5.0, math.pi / 2, math.pi / 2, 2.0 * math.pi / 3.0)


def unit_atoms() -> Atoms:
    """One atom at the origin with f(s) = 1 (all Gaussian amplitudes zero,
    constant 1), B = 0 and occupancy 1: F_hkl = 1 for every reflection."""
    ff = np.zeros((1, 9))
    ff[0, 4:8] = 1.0
    ff[0, 8] = 1.0
    return Atoms(frac=np.zeros((1, 3)), B=np.zeros(1), occ=np.ones(1), elem=np.zeros(1, np.uint8), ff=ff)


def gvl(kind: str, n_px: int = 511, n_nodes: int = 64, L: float = 150.0) -> Problem:
    """Fig. GvL: Gaussian (sigma = 3 deg, gamma = 0) or Lorentzian (sigma = 0,
    gamma = 3 deg) orientation distribution, |F| = 1, Hosemann lineshape with
    no paracrystal term (g = 0), d >= 2 A, square detector of n_px 0.2 mm
    pixels at the distance of Eq. SF for 2 A."""
    if kind not in ("gauss", "lorentz"):
        raise ValueError("kind is 'gauss' or 'lorentz'")
    sig, gam = (math.radians(3.0), 0.0) if kind == "gauss" else (0.0, math.radians(3.0))
    br = Broadening(L=(L, L, L), g=(0.0, 0.0, 0.0), lineshape=LINESHAPE_HOSEMANN,
                    intensity_model=INTENSITY_HOSEMANN, sigma=sig, gamma=gam, T=patch_extent(sig, gam),
                    n_nodes=n_nodes)
    pix = 0.2
    geom = Geometry(wavelength=1.0, distance=distance_for_resolution(n_px, pix, 1.0, 2.0), pixel=pix,
                    n_x=n_px, n_y=n_px)
    return Problem("gvl_" + kind, FIGURE_CELL, unit_atoms(), 2.0, 0.0, br, geom, 0)


def equator(g: float, B: float, n_x: int = 1023, n_y: int = 15, n_nodes: int = 48, L: float = 150.0) -> Problem:
    """Fig. equator: |F| = 1 with isotropic paracrystal disorder g_a = g_b =
    g_c = g and isotropic axis Debye-Waller B_a = B_b = B_c = B, Gaussian
    orientation sigma = 2 deg, d >= 2 A.  A strip of n_x x n_y 0.1 mm pixels
    (n_y odd: the middle row lies on the equator) at the distance of Eq. SF
    for 2 A across n_x pixels."""
    if n_y % 2 == 0:
        raise ValueError("n_y must be odd")
    sig = math.radians(2.0)
    br = Broadening(L=(L, L, L), g=(g, g, g), B_axis=(B, B, B), lineshape=LINESHAPE_HOSEMANN,
                    intensity_model=INTENSITY_HOSEMANN, sigma=sig, gamma=0.0, T=patch_extent(sig, 0.0),
                    n_nodes=n_nodes)
    pix = 0.1
    geom = Geometry(wavelength=1.0, distance=distance_for_resolution(n_x, pix, 1.0, 2.0), pixel=pix,
                    n_x=n_x, n_y=n_y)
    return Problem("equator_g%g_B%g" % (g, B), FIGURE_CELL, unit_atoms(), 2.0, 0.0, br, geom, 0)


CONFIGS = {
    0: config0,
    1: config1,
    2: config2,
}
