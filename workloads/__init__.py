"""Seeded synthetic inputs for the multibody axisymmetric sound-soft scattering problem.

This module only draws and lays out inputs: shape descriptions, body centres and
orientations, wave parameters, incident plane-wave directions, interior point sources
and exterior target points.  It contains no arithmetic of the solution method
(no quadrature, no kernel, no discretisation), so both the CUDA path and the
independent oracle can read the same inputs without sharing any method code.

The paper (Hao, Martinsson, Young, Sec. 6) measures accuracy with one random point
source inside each body and an exact exterior solution evaluated at 10 random
targets a few wavelengths out; `point_sources` and `exterior_targets` draw those.
Its geometries are given only as figures, so the named workloads below are
synthetic stand-ins with the body counts, sizes and wavenumbers stated in each
function.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np
from scipy.spatial import cKDTree

SPHERE = 0
SPHEROID = 1
OPEN_SHELL = 2
CURVE_SPLINE = 3

DEFAULT_SEED = 20140601


@dataclass(frozen=True)
class ShapeSpec:
    """A rotationally symmetric body in its own frame (symmetry axis = body z).

    kind SPHERE:     params = (a,)                 radius a
    kind SPHEROID:   params = (a, c)               semi-axes (a, a, c)
    kind OPEN_SHELL: params = (R_out, R_in, half_angle_rad, rim_radius)
                     a thick spherical shell whose opening (centred on body -z)
                     has the given half-angle; the rim is a semicircle.
    kind CURVE_SPLINE: params = (r_0, z_0, r_1, z_1, ...), the points of a cubic-spline
                     generating curve from the top pole (r_0 = 0) to the bottom pole;
                     n_panels must equal the number of points - 1 (one panel per segment).
    n_panels Gauss-Legendre panels of gl_order nodes each on the generating
    curve, n_modes (odd) equispaced azimuthal nodes.
    """
    kind: int
    params: tuple
    n_panels: int
    gl_order: int
    n_modes: int

    @property
    def n_rings(self) -> int:
        return self.n_panels * self.gl_order

    @property
    def n_nodes(self) -> int:
        return self.n_rings * self.n_modes

    def bounding_radius(self) -> float:
        if self.kind == SPHERE:
            return float(self.params[0])
        if self.kind == SPHEROID:
            return float(max(self.params[0], self.params[1]))
        if self.kind == CURVE_SPLINE:
            rz = np.asarray(self.params, dtype=float).reshape(-1, 2)
            return float(np.max(np.hypot(rz[:, 0], rz[:, 1])) * 1.05)
        return float(self.params[0])

    def curve_points(self) -> np.ndarray:
        """(n, 2) array of (r, z) points of a CURVE_SPLINE shape."""
        return np.asarray(self.params, dtype=float).reshape(-1, 2)


@dataclass
class Body:
    shape: ShapeSpec
    center: np.ndarray          # (3,)
    rot: np.ndarray             # (3,3): columns are the body x, y, z axes in world coordinates


@dataclass
class Workload:
    name: str
    bodies: List[Body]
    k: float
    eta: float
    directions: np.ndarray      # (R,3) unit incident directions
    gmres_tol: float = 1e-10
    extra: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return sum(b.shape.n_nodes for b in self.bodies)

    @property
    def n_rhs(self) -> int:
        return int(self.directions.shape[0])

    def distinct_shapes(self) -> List[ShapeSpec]:
        out: List[ShapeSpec] = []
        for b in self.bodies:
            if b.shape not in out:
                out.append(b.shape)
        return out


def rotation_taking_z_to(a) -> np.ndarray:
    """Smallest rotation taking e_z to the unit vector a (Rodrigues about e_z x a).

    When a is (numerically) -e_z the rotation is a half turn about e_x.
    Returned as a 3x3 matrix whose columns are the images of e_x, e_y, e_z.
    """
    a = np.asarray(a, dtype=np.float64)
    a = a / np.linalg.norm(a)
    ez = np.array([0.0, 0.0, 1.0])
    c = float(a @ ez)
    if c < -1.0 + 1e-12:
        return np.diag([1.0, -1.0, -1.0])
    v = np.cross(ez, a)
    vx = np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])
    return np.eye(3) + vx + vx @ vx / (1.0 + c)


def uniform_directions(n: int, seed: int) -> np.ndarray:
    """n directions uniform on the unit sphere (normalised Gaussian vectors)."""
    g = np.random.default_rng(seed).standard_normal((n, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def _surface_samples(body: Body, n: int = 1500) -> np.ndarray:
    """Points on a conservative outer envelope of a body, for the gap check only.

    Sphere and spheroid: the surface itself.  Open shell: its outer sphere, which
    contains the whole shell.  Fibonacci points in the body frame, mapped to world.
    """
    i = np.arange(n) + 0.5
    ct = 1.0 - 2.0 * i / n
    st = np.sqrt(1.0 - ct * ct)
    ph = np.pi * (1.0 + 5.0 ** 0.5) * i
    u = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    s = body.shape
    if s.kind == SPHERE:
        p = s.params[0] * u
    elif s.kind == SPHEROID:
        p = u * np.array([s.params[0], s.params[0], s.params[1]])
    else:
        p = s.params[0] * u
    return p @ body.rot.T + body.center


def gap_to(bodies: List[Body], cand: Body, samples=None) -> float:
    """Smallest envelope distance between `cand` and any of `bodies`."""
    pc = _surface_samples(cand)
    best = np.inf
    for q, b in enumerate(bodies):
        if np.linalg.norm(b.center - cand.center) > b.shape.bounding_radius() + cand.shape.bounding_radius() + best:
            continue
        pb = samples[q] if samples is not None else _surface_samples(b)
        best = min(best, float(cKDTree(pb).query(pc)[0].min()))
    return best


def min_gap(bodies: List[Body]) -> float:
    pts = [_surface_samples(b) for b in bodies]
    best = np.inf
    for a in range(len(bodies)):
        for b in range(a + 1, len(bodies)):
            if np.linalg.norm(bodies[a].center - bodies[b].center) > (
                    bodies[a].shape.bounding_radius() + bodies[b].shape.bounding_radius() + best):
                continue
            d = np.sqrt(((pts[a][:, None, :] - pts[b][None, :, :]) ** 2).sum(-1)).min()
            best = min(best, float(d))
    return best


# --------------------------------------------------------------------------- workloads

def pear_curve(n_points: int = 13, a: float = 1.0, e: float = 0.25) -> tuple:
    """Points (r, z) of an egg/pear-shaped generating curve, rho(th) = a (1 + e cos th)
    sampled at equal polar angles th from 0 (top pole) to pi (bottom pole); a
    CURVE_SPLINE shape interpolates them with one panel per segment."""
    th = np.linspace(0.0, np.pi, n_points)
    rho = a * (1.0 + e * np.cos(th))
    r = rho * np.sin(th)
    r[0] = 0.0
    r[-1] = 0.0
    z = rho * np.cos(th)
    return tuple(np.stack([r, z], axis=1).reshape(-1).tolist())


def two_spheres(n_panels=10, gl_order=10, n_modes=41, k=2.0, eta=None, sep=1.5,
                directions=None, name="two_spheres_8200") -> Workload:
    """Two sound-soft unit spheres centred at (+-sep, 0, 0); k = eta = 2; 10 x 10 GL
    nodes on the generating semicircle and 41 azimuthal nodes: 8,200 unknowns.
    Plane wave along +z."""
    shape = ShapeSpec(SPHERE, (1.0,), n_panels, gl_order, n_modes)
    bodies = [Body(shape, np.array([-sep, 0.0, 0.0]), np.eye(3)),
              Body(shape, np.array([+sep, 0.0, 0.0]), np.eye(3))]
    if directions is None:
        directions = np.array([[0.0, 0.0, 1.0]])
    return Workload(name, bodies, k, k if eta is None else eta, np.asarray(directions, float),
                    gmres_tol=1e-10)


def tiny_two_spheres(n_panels=4, gl_order=6, n_modes=9, k=1.0, sep=1.6) -> Workload:
    """A small two-sphere case (432 unknowns) that the oracle finishes in seconds."""
    return two_spheres(n_panels, gl_order, n_modes, k=k, sep=sep, name="two_spheres_tiny")


def separated_spheroids(n_bodies=3, spacing=3.5, a=0.5, c=1.0, n_panels=4, gl_order=6, n_modes=11,
                        k=2.0, seed=DEFAULT_SEED, name="separated_spheroids") -> Workload:
    """n_bodies spheroids (a, a, c) with seeded random symmetry axes, centres on a line
    along x with the given spacing plus a seeded transverse jitter of 0.3 spacing; for
    the accelerated scheme (Sec. 5), whose compression needs bodies that are not tightly
    packed.  Plane wave along +z."""
    rng = np.random.default_rng(seed)
    shape = ShapeSpec(SPHEROID, (a, c), n_panels, gl_order, n_modes)
    bodies = []
    for q in range(n_bodies):
        cen = np.array([spacing * q, 0.0, 0.0])
        cen[1:] += 0.3 * spacing * (rng.random(2) - 0.5)
        bodies.append(Body(shape, cen, rotation_taking_z_to(rng.standard_normal(3))))
    return Workload(name, bodies, k, k, np.array([[0.0, 0.0, 1.0]]), gmres_tol=1e-10)


def spheroids8(seed=DEFAULT_SEED, n_panels=20, gl_order=16, n_modes=101, k=4.0,
               n_rhs=1) -> Workload:
    """Eight prolate spheroids, semi-axes (1,1,2), symmetry axes uniform on the sphere
    (seeded), centres on a 2x2x2 grid of spacing 5; k = eta = 4; 20 panels x 16 GL
    nodes and 101 azimuthal nodes per body: 258,560 unknowns.  One plane wave
    along +z by default."""
    rng = np.random.default_rng(seed)
    shape = ShapeSpec(SPHEROID, (1.0, 2.0), n_panels, gl_order, n_modes)
    axes = rng.standard_normal((8, 3))
    bodies = []
    idx = 0
    for ix in range(2):
        for iy in range(2):
            for iz in range(2):
                c = 5.0 * np.array([ix, iy, iz], float) - 2.5
                bodies.append(Body(shape, c, rotation_taking_z_to(axes[idx])))
                idx += 1
    dirs = np.array([[0.0, 0.0, 1.0]]) if n_rhs == 1 else uniform_directions(n_rhs, seed + 1)
    return Workload("spheroids8_258560", bodies, k, k, dirs, gmres_tol=1e-10)


def mixed27(seed=DEFAULT_SEED, n_rhs=64, k=4.0) -> Workload:
    """27 bodies on a 3x3x3 grid of spacing 5: a seeded 50/50 mix of spheres
    (radius U[0.5,1.5]) and spheroids (1,1,c), c ~ U[1,2]; each body draws its own
    panel count in [12,24] (16 GL nodes each) and odd azimuthal count in [61,121];
    k = eta = 4; 64 plane waves uniform on the sphere."""
    rng = np.random.default_rng(seed)
    bodies = []
    for ix in range(3):
        for iy in range(3):
            for iz in range(3):
                c = 5.0 * np.array([ix, iy, iz], float) - 5.0
                npan = int(rng.integers(12, 25))
                nf = int(2 * rng.integers(30, 61) + 1)
                if rng.random() < 0.5:
                    shape = ShapeSpec(SPHERE, (float(rng.uniform(0.5, 1.5)),), npan, 16, nf)
                    rot = np.eye(3)
                else:
                    shape = ShapeSpec(SPHEROID, (1.0, float(rng.uniform(1.0, 2.0))), npan, 16, nf)
                    rot = rotation_taking_z_to(rng.standard_normal(3))
                bodies.append(Body(shape, c, rot))
    return Workload("mixed27", bodies, k, k, uniform_directions(n_rhs, seed + 7), gmres_tol=1e-10)


def mixed48(seed=DEFAULT_SEED, n_rhs=16, k=6.0, n_panels=24, gl_order=16, n_modes=121,
            min_gap_required=1.0) -> Workload:
    """48 bodies on a jittered 4x4x3 grid (spacing 4.5, jitter U[-0.5,0.5]^3 per centre):
    16 unit spheres, 16 spheroids (1,1,2), 16 open shells (outer radius 1, inner 0.8,
    opening half-angle 60 degrees, rim semicircle radius 0.1), seeded orientations,
    redrawn until every surface gap is at least 1; k = eta = 6; 24 panels x 16 GL
    nodes and 121 azimuthal nodes per body (about 2.2 M unknowns); 16 plane waves."""
    rng = np.random.default_rng(seed)
    kinds = np.array([SPHERE] * 16 + [SPHEROID] * 16 + [OPEN_SHELL] * 16)
    rng.shuffle(kinds)
    shapes = {
        SPHERE: ShapeSpec(SPHERE, (1.0,), n_panels, gl_order, n_modes),
        SPHEROID: ShapeSpec(SPHEROID, (1.0, 2.0), n_panels, gl_order, n_modes),
        OPEN_SHELL: ShapeSpec(OPEN_SHELL, (1.0, 0.8, np.pi / 3.0, 0.1), n_panels, gl_order, n_modes),
    }
    bodies: List[Body] = []
    samples = []
    idx = 0
    for ix in range(4):
        for iy in range(4):
            for iz in range(3):
                base = 4.5 * np.array([ix - 1.5, iy - 1.5, iz - 1.0])
                for _attempt in range(200):
                    c = base + rng.uniform(-0.5, 0.5, 3)
                    rot = rotation_taking_z_to(rng.standard_normal(3))
                    cand = Body(shapes[int(kinds[idx])], c, rot)
                    # placed bodies already keep the gap among themselves
                    if not bodies or gap_to(bodies, cand, samples) >= min_gap_required:
                        break
                else:
                    raise RuntimeError("could not place body %d with the required gap" % idx)
                bodies.append(cand)
                samples.append(_surface_samples(cand))
                idx += 1
    return Workload("mixed48_shells", bodies, k, k, uniform_directions(n_rhs, seed + 11),
                    gmres_tol=1e-10)


def mixed4_shells(seed=DEFAULT_SEED, n_rhs=2, k=6.0, n_panels=12, gl_order=10, n_modes=61,
                  min_gap_required=1.0) -> Workload:
    """A reduced form of the 48-body workload that the oracle solves in minutes: a unit
    sphere, a spheroid (1,1,2) and two open shells (1, 0.8, 60 degrees, rim 0.1) on a
    jittered 2x2x1 grid of spacing 4.5 (jitter U[-0.5,0.5]^3, seeded orientations,
    surface gaps >= 1); k = eta = 6; 12 panels x gl_order GL nodes and 61 azimuthal
    nodes per body; n_rhs plane waves uniform on the sphere."""
    rng = np.random.default_rng(seed + 5)
    shapes = [ShapeSpec(SPHERE, (1.0,), n_panels, gl_order, n_modes),
              ShapeSpec(SPHEROID, (1.0, 2.0), n_panels, gl_order, n_modes),
              ShapeSpec(OPEN_SHELL, (1.0, 0.8, np.pi / 3.0, 0.1), n_panels, gl_order, n_modes),
              ShapeSpec(OPEN_SHELL, (1.0, 0.8, np.pi / 3.0, 0.1), n_panels, gl_order, n_modes)]
    bodies: List[Body] = []
    samples = []
    for idx, (ix, iy) in enumerate([(0, 0), (1, 0), (0, 1), (1, 1)]):
        base = 4.5 * np.array([ix - 0.5, iy - 0.5, 0.0])
        for _attempt in range(200):
            cand = Body(shapes[idx], base + rng.uniform(-0.5, 0.5, 3), rotation_taking_z_to(rng.standard_normal(3)))
            if not bodies or gap_to(bodies, cand, samples) >= min_gap_required:
                break
        else:
            raise RuntimeError("could not place body %d with the required gap" % idx)
        bodies.append(cand)
        samples.append(_surface_samples(cand))
    return Workload("mixed4_shells", bodies, k, k, uniform_directions(n_rhs, seed + 13), gmres_tol=1e-10)


def uneven3(seed=DEFAULT_SEED, n_rhs=8, k=4.0) -> Workload:
    """A reduced form of the 27-body workload: three bodies on a line of spacing 5, a
    seeded mix of spheres (radius U[0.5,1.5]) and spheroids (1,1,c), c ~ U[1,2], each
    with its own panel count in [6,12] (8 GL nodes each) and odd azimuthal count in
    [21,41] (uneven sizes); k = eta = 4; n_rhs plane waves uniform on the sphere,
    solved as one batch."""
    rng = np.random.default_rng(seed + 3)
    bodies = []
    kinds = [SPHERE, SPHEROID, SPHEROID]
    for q in range(3):
        npan = int(rng.integers(6, 13))
        nf = int(2 * rng.integers(10, 21) + 1)
        c = np.array([5.0 * (q - 1), 0.0, 0.0]) + rng.uniform(-0.5, 0.5, 3)
        if kinds[q] == SPHERE:
            shape = ShapeSpec(SPHERE, (float(rng.uniform(0.5, 1.5)),), npan, 8, nf)
            rot = np.eye(3)
        else:
            shape = ShapeSpec(SPHEROID, (1.0, float(rng.uniform(1.0, 2.0))), npan, 8, nf)
            rot = rotation_taking_z_to(rng.standard_normal(3))
        bodies.append(Body(shape, c, rot))
    return Workload("uneven3", bodies, k, k, uniform_directions(n_rhs, seed + 17), gmres_tol=1e-10)


def point_sources(wl: Workload, seed: int) -> np.ndarray:
    """One point source inside each body (world coordinates), as in the paper's
    accuracy protocol (Sec. 6).  Spheres and spheroids: centre plus 0.3 x (smallest
    semi-axis) x a uniform point of the unit ball.  Open shells (whose centre is
    cavity fluid): inside the wall at body-frame radius 0.9 x R_out, polar angle in
    [10, 100] degrees, azimuth uniform."""
    rng = np.random.default_rng(seed)
    out = []
    for b in wl.bodies:
        s = b.shape
        if s.kind in (SPHERE, SPHEROID):
            g = rng.standard_normal(3)
            g /= np.linalg.norm(g)
            rad = 0.3 * min(s.params) * rng.random() ** (1.0 / 3.0)
            p = rad * g
        else:
            rho = 0.5 * (s.params[0] + s.params[1])
            th = np.deg2rad(rng.uniform(10.0, 100.0))
            ph = rng.uniform(0.0, 2.0 * np.pi)
            p = rho * np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        out.append(b.center + b.rot @ p)
    return np.array(out)


def exterior_targets(wl: Workload, n: int, seed: int, wavelengths: float = 3.0) -> np.ndarray:
    """n points uniform on the sphere of radius R_encl + wavelengths * (2 pi / k) about
    the centroid of the body centres; R_encl encloses every body."""
    cen = np.mean([b.center for b in wl.bodies], axis=0)
    r_encl = max(np.linalg.norm(b.center - cen) + b.shape.bounding_radius() for b in wl.bodies)
    rad = r_encl + wavelengths * 2.0 * np.pi / wl.k
    return cen + rad * uniform_directions(n, seed)


def by_name(name: str, **kw) -> Workload:
    table = {
        "two_spheres_8200": two_spheres,
        "two_spheres_tiny": tiny_two_spheres,
        "spheroids8_258560": spheroids8,
        "mixed27": mixed27,
        "mixed48_shells": mixed48,
        "mixed4_shells": mixed4_shells,
        "uneven3": uneven3,
    }
    return table[name](**kw)
