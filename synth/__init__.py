"""Seeded synthetic surfaces and boundary data for the FMM-LU workloads.

This module is shared by the tests, the benchmark and the oracle's callers. It
holds only input generation: point clouds on closed surfaces with unit outward
normals and quadrature weights, and incident-field boundary data. It holds none
of the solver's arithmetic (no system matrix, no compression, no elimination).

The paper measures on wiggly tori and an aircraft mesh discretised with
high-order patches (Sec. 6, Eq. wtorus); those meshes and their quadrature are
not available, so these smooth closed surfaces stand in for them with the same
role: multiscale closed surfaces one to twenty wavelengths across.

Every generator is deterministic in its arguments (numpy ``default_rng(seed)``).
Arrays are float64, points/normals shaped (N, 3), weights (N,).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))


@dataclass
class Surface:
    """A sampled closed surface: nodes, unit outward normals, area weights."""

    points: np.ndarray
    normals: np.ndarray
    weights: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.points.shape[0])


# ---------------------------------------------------------------------------
# point sets on the unit sphere
# ---------------------------------------------------------------------------

def fibonacci_unit(n: int) -> np.ndarray:
    """Fibonacci lattice on the unit sphere: z_i = 1-(2i+1)/n, phi_i = i*golden."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * GOLDEN_ANGLE
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def sphere_fibonacci(n: int, radius: float = 1.0) -> Surface:
    """Sphere of the given radius; weights 4 pi r^2 / n; normals = positions / r."""
    u = fibonacci_unit(n)
    w = np.full(n, 4.0 * math.pi * radius * radius / n)
    return Surface(points=radius * u, normals=u.copy(), weights=w,
                   name=f"sphere_fib_{n}")


def _uniform_directions(rng: np.random.Generator, m: int) -> np.ndarray:
    g = rng.standard_normal((m, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


# ---------------------------------------------------------------------------
# ellipsoids
# ---------------------------------------------------------------------------

def _ellipsoid_jacobian(u: np.ndarray, axes) -> np.ndarray:
    """Area ratio dA_ellipsoid / dA_sphere of the map u -> (a u1, b u2, c u3)."""
    a, b, c = axes
    return a * b * c * np.sqrt((u[:, 0] / a) ** 2 + (u[:, 1] / b) ** 2
                               + (u[:, 2] / c) ** 2)


def _sphere_quadrature(nt: int = 256, nphi: int = 512):
    """Gauss-Legendre in cos(theta) x trapezoid in phi on the unit sphere."""
    x, wx = np.polynomial.legendre.leggauss(nt)
    phi = (np.arange(nphi) + 0.5) * (2.0 * math.pi / nphi)
    ct = np.repeat(x, nphi)
    st = np.sqrt(1.0 - ct * ct)
    ph = np.tile(phi, nt)
    u = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    wq = np.repeat(wx, nphi) * (2.0 * math.pi / nphi)
    return u, wq


def ellipsoid_area(axes) -> float:
    u, wq = _sphere_quadrature()
    return float(np.sum(wq * _ellipsoid_jacobian(u, axes)))


def _ellipsoid_normals(p: np.ndarray, axes) -> np.ndarray:
    a, b, c = axes
    nv = np.stack([p[:, 0] / a ** 2, p[:, 1] / b ** 2, p[:, 2] / c ** 2], axis=1)
    return nv / np.linalg.norm(nv, axis=1, keepdims=True)


def ellipsoid_uniform(n: int, axes=(1.0, 2.0, 0.5), seed: int = 2202) -> Surface:
    """Area-uniform random points on an ellipsoid, weights area/n.

    Directions u are uniform on the sphere, mapped to (a u1, b u2, c u3) and
    accepted with probability proportional to the area Jacobian.
    """
    rng = np.random.default_rng(seed)
    jmax = float(np.prod(axes)) / min(axes)
    out = []
    have = 0
    while have < n:
        m = max(1024, 2 * (n - have))
        u = _uniform_directions(rng, m)
        acc = rng.random(m) * jmax < _ellipsoid_jacobian(u, axes)
        u = u[acc]
        out.append(u)
        have += u.shape[0]
    u = np.concatenate(out)[:n]
    p = u * np.asarray(axes)[None, :]
    area = ellipsoid_area(axes)
    return Surface(points=p, normals=_ellipsoid_normals(p, axes),
                   weights=np.full(n, area / n),
                   name=f"ellipsoid{tuple(axes)}_{n}")


def ellipsoid_graded_tip(n: int, axes=(1.0, 3.0, 0.5), ratio: float = 100.0,
                         seed: int = 2205) -> Surface:
    """Ellipsoid sampled with density proportional to 1/max(theta, theta0).

    theta is the angle between the sphere direction u and the +y axis and
    theta0 = pi/ratio, so the density is `ratio` times higher at the +y tip than
    at the opposite tip. Weights are importance weights Z/(n f(x)).
    """
    rng = np.random.default_rng(seed)
    th0 = math.pi / ratio
    jmax = float(np.prod(axes)) / min(axes)

    def dens(u):
        th = np.arccos(np.clip(u[:, 1], -1.0, 1.0))
        return 1.0 / np.maximum(th, th0)

    fmax = 1.0 / th0
    out = []
    have = 0
    while have < n:
        m = max(4096, 8 * (n - have))
        u = _uniform_directions(rng, m)
        acc = rng.random(m) * jmax < _ellipsoid_jacobian(u, axes)
        u = u[acc]
        acc2 = rng.random(u.shape[0]) * fmax < dens(u)
        u = u[acc2]
        out.append(u)
        have += u.shape[0]
    u = np.concatenate(out)[:n]
    p = u * np.asarray(axes)[None, :]
    uq, wq = _sphere_quadrature(512, 1024)
    z = float(np.sum(wq * _ellipsoid_jacobian(uq, axes) * dens(uq)))
    w = z / (n * dens(u))
    return Surface(points=p, normals=_ellipsoid_normals(p, axes), weights=w,
                   name=f"ellipsoid_graded{tuple(axes)}_{n}")


# ---------------------------------------------------------------------------
# torus graded toward one meridian
# ---------------------------------------------------------------------------

def torus_graded(n: int, R: float = 2.0, r: float = 0.5, ratio: float = 1000.0,
                 seed: int = 2203) -> Surface:
    """Torus with toroidal-angle density proportional to 1/max(|u|, pi/ratio).

    u in [-pi, pi) by inverse CDF (log-uniform away from the u = 0 meridian),
    poloidal angle v with density proportional to R + r cos v by rejection.
    Weights are the importance weights r (R + r cos v) / (n p(u) p(v)).
    """
    rng = np.random.default_rng(seed)
    u0 = math.pi / ratio
    c = 1.0 + math.log(math.pi / u0)          # integral of f over [0, pi]
    t = rng.random(n) * c
    au = np.where(t <= 1.0, t * u0, u0 * np.exp(t - 1.0))
    sgn = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    uu = sgn * au
    pu = 1.0 / np.maximum(np.abs(uu), u0) / (2.0 * c)
    v = np.empty(n)
    have = 0
    while have < n:
        m = 2 * (n - have) + 64
        cand = rng.random(m) * 2.0 * math.pi
        acc = rng.random(m) * (R + r) < R + r * np.cos(cand)
        cand = cand[acc][: n - have]
        v[have:have + cand.shape[0]] = cand
        have += cand.shape[0]
    pv = (R + r * np.cos(v)) / (2.0 * math.pi * R)
    rho = R + r * np.cos(v)
    p = np.stack([rho * np.cos(uu), rho * np.sin(uu), r * np.sin(v)], axis=1)
    nv = np.stack([np.cos(v) * np.cos(uu), np.cos(v) * np.sin(uu), np.sin(v)],
                  axis=1)
    w = r * rho / (n * pu * pv)
    return Surface(points=p, normals=nv, weights=w, name=f"torus_graded_{n}")


# ---------------------------------------------------------------------------
# boundary data (incident fields); sound-soft scattering uses f = -u_inc
# ---------------------------------------------------------------------------

def point_source_field(x: np.ndarray, src, k: float) -> np.ndarray:
    """Field of a unit point source at `src`: exp(i k r)/(4 pi r)."""
    d = np.linalg.norm(x - np.asarray(src, dtype=np.float64)[None, :], axis=1)
    return np.exp(1j * k * d) / (4.0 * math.pi * d)


def plane_wave(x: np.ndarray, direction, k: float) -> np.ndarray:
    """Incident plane wave exp(i k d.x) for a unit direction d."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.exp(1j * k * (x @ d))


def seeded_directions(m: int, seed: int) -> np.ndarray:
    """m unit directions from normalised Gaussians."""
    return _uniform_directions(np.random.default_rng(seed), m)


def scaled_rhs(surface: Surface, f: np.ndarray) -> np.ndarray:
    """Right-hand side of the sqrt(w)-scaled system: b = sqrt(w) f."""
    s = np.sqrt(surface.weights)
    return s[:, None] * f if f.ndim == 2 else s * f


def exterior_targets(m: int, radius: float = 3.0) -> np.ndarray:
    return radius * fibonacci_unit(m)


# ---------------------------------------------------------------------------
# the named workloads
# ---------------------------------------------------------------------------

WORKLOADS = {
    # name: (builder, k, eps)
    "sphere2k": dict(n=2000, k=1.0, eps=1e-6),
    "ellipsoid50k": dict(n=50000, k=2.0 * math.pi, eps=1e-6),
    "torus200k": dict(n=200000, k=5.0, eps=1e-4),
    "sphere100k": dict(n=100000, k=10.0, eps=1e-6),
    "ellipsoid1m": dict(n=1000000, k=20.0, eps=1e-4),
    # azimuthal sonar sweep (Sec. 6.3) on a multiscale surface: 128 incident
    # directions (cos phi, sin phi, 0), phi uniform in [0, 2 pi)
    "sonar200k": dict(n=200000, k=10.0, eps=1e-4, angles=128),
}


def azimuthal_angles(m: int) -> np.ndarray:
    """m incidence angles phi_j = 2 pi j / m of an azimuthal sweep."""
    return 2.0 * math.pi * np.arange(m) / m


def make_surface(name: str, n: int | None = None) -> Surface:
    """Build the surface of a named workload (optionally at another size)."""
    spec = WORKLOADS[name]
    n = spec["n"] if n is None else n
    if name in ("sphere2k", "sphere100k"):
        return sphere_fibonacci(n)
    if name == "ellipsoid50k":
        return ellipsoid_uniform(n, (1.0, 2.0, 0.5), seed=2202)
    if name == "torus200k":
        return torus_graded(n, seed=2203)
    if name == "ellipsoid1m":
        return ellipsoid_graded_tip(n, (1.0, 3.0, 0.5), seed=2205)
    if name == "sonar200k":
        return ellipsoid_graded_tip(n, (1.0, 3.0, 0.5), seed=2206)
    raise KeyError(name)


def make_rhs(name: str, surface: Surface, k: float | None = None) -> np.ndarray:
    """Scaled right-hand side(s) b = sqrt(w) f of a named workload."""
    spec = WORKLOADS[name]
    k = spec["k"] if k is None else k
    x = surface.points
    if name == "sphere2k":
        return scaled_rhs(surface, point_source_field(x, (0.1, 0.2, -0.1), k))
    if name == "ellipsoid50k":
        return scaled_rhs(surface, -plane_wave(x, (0.0, 0.0, 1.0), k))
    if name == "torus200k":
        return scaled_rhs(surface, -plane_wave(x, (0.0, 0.0, 1.0), k))
    if name == "sphere100k":
        dirs = seeded_directions(64, 2204)
        f = np.stack([-plane_wave(x, d, k) for d in dirs], axis=1)
        return scaled_rhs(surface, f)
    if name == "ellipsoid1m":
        dirs = seeded_directions(16, 2205)
        f = np.stack([-plane_wave(x, d, k) for d in dirs], axis=1)
        return scaled_rhs(surface, f)
    if name == "sonar200k":
        ph = azimuthal_angles(spec["angles"])
        dirs = np.stack([np.cos(ph), np.sin(ph), np.zeros_like(ph)], axis=1)
        f = np.stack([-plane_wave(x, d, k) for d in dirs], axis=1)
        return scaled_rhs(surface, f)
    raise KeyError(name)
