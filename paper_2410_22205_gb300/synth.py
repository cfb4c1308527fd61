"""Seeded synthetic inputs: point clouds, grids and initial level sets.

This module holds no arithmetic of the reconstruction method itself. It only
draws inputs: point clouds shaped like the paper's test objects (§4: circle,
sphere, torus-like and scan-like clouds), uniform Cartesian grids, and the
analytic initial level sets the workloads prescribe. Both the CUDA path and
the FP64 oracle consume these arrays; neither imports the other.

Every generator takes an explicit seed and uses numpy's PCG64 generator, so
the same call gives the same bytes on x86 and Arm hosts.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Grid:
    """Uniform Cartesian grid: ``n`` nodes per axis on the box [lo, hi].

    Both end points are nodes, so the mesh width is (hi - lo) / (n - 1) and
    must be equal on every axis (§3: one mesh width Δx for the whole grid).
    In 2-D the third axis has one node.
    """

    dim: int
    n: tuple
    lo: tuple
    hi: tuple

    @property
    def h(self) -> float:
        return (self.hi[0] - self.lo[0]) / (self.n[0] - 1)

    @property
    def num_nodes(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    def axes(self):
        """Node coordinates per axis, computed as lo + i*h in FP64."""
        h = self.h
        return [self.lo[a] + np.arange(self.n[a], dtype=np.float64) * h for a in range(self.dim)]


def cube_grid(dim: int, n: int, lo: float = -1.0, hi: float = 1.0) -> Grid:
    if dim == 2:
        return Grid(2, (n, n, 1), (lo, lo, 0.0), (hi, hi, 0.0))
    return Grid(3, (n, n, n), (lo, lo, lo), (hi, hi, hi))


def sphere_sdf(grid: Grid, radius: float, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Signed distance |x - c| - r to a circle/sphere, on every node.

    Returned flat in the grid's linear order (x fastest). This is the initial
    level set the workloads prescribe (a circle of radius 0.9 in 2-D, a sphere
    of radius 0.9 in 3-D); it is an input, not part of the method.
    """
    ax = grid.axes()
    if grid.dim == 2:
        y, x = np.meshgrid(ax[1], ax[0], indexing="ij")
        r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2)
    else:
        z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    return (r - radius).reshape(-1)


# --------------------------------------------------------------------------
# Point clouds
# --------------------------------------------------------------------------

def circle_uniform(n: int = 64, radius: float = 1.0) -> np.ndarray:
    """n points at equal angles on a circle (the paper's 2-D circle test, §4.1)."""
    t = 2.0 * np.pi * np.arange(n) / n
    return np.stack([radius * np.cos(t), radius * np.sin(t)], axis=1)


def circle_noisy(n: int = 200, radius: float = 0.5, sigma: float = 0.005, seed: int = 0) -> np.ndarray:
    """Uniform angle, Gaussian radial noise: the small 2-D workload (64^2 grid)."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.0, 2.0 * np.pi, n)
    r = radius + rng.normal(0.0, sigma, n)
    return np.stack([r * np.cos(t), r * np.sin(t)], axis=1)


def circle_even_noisy(n: int = 600, radius: float = 0.5, sigma: float = 0.002, seed: int = 0) -> np.ndarray:
    """Equal angles, Gaussian radial noise: a scan of a circle without holes."""
    rng = np.random.default_rng(seed)
    t = 2.0 * np.pi * np.arange(n) / n
    r = radius + rng.normal(0.0, sigma, n)
    return np.stack([r * np.cos(t), r * np.sin(t)], axis=1)


def torus_cloud(n: int = 20000, R: float = 0.5, r: float = 0.2, sigma: float = 0.002, seed: int = 1) -> np.ndarray:
    """Area-uniform torus samples with Gaussian displacement along the normal.

    Area uniformity: the torus area element is proportional to (R + r cos v),
    so v is drawn by rejection against (R + r cos v) / (R + r).
    """
    rng = np.random.default_rng(seed)
    out = []
    have = 0
    while have < n:
        m = 2 * (n - have) + 1024
        v = rng.uniform(0.0, 2.0 * np.pi, m)
        keep = rng.uniform(0.0, 1.0, m) < (R + r * np.cos(v)) / (R + r)
        v = v[keep]
        u = rng.uniform(0.0, 2.0 * np.pi, v.size)
        eps = rng.normal(0.0, sigma, v.size)
        rr = r + eps
        x = (R + rr * np.cos(v)) * np.cos(u)
        y = (R + rr * np.cos(v)) * np.sin(u)
        z = rr * np.sin(v)
        out.append(np.stack([x, y, z], axis=1))
        have += v.size
    return np.concatenate(out)[:n]


def sphere_cloud(n: int, radius: float = 1.0, sigma: float = 0.0, seed: int = 0, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Uniform points on a sphere (normalised Gaussian directions)."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    rr = radius + (rng.normal(0.0, sigma, n) if sigma > 0 else 0.0)
    return v * np.asarray(rr).reshape(-1, 1) + np.asarray(center)


def sphere_even(n: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n evenly spread points on a sphere (the golden-angle spiral: equal-area
    latitude bands, longitude advancing by the golden angle), a stand-in for
    a scan without holes."""
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    t = np.pi * (3.0 - np.sqrt(5.0)) * np.arange(n)
    v = np.stack([r * np.cos(t), r * np.sin(t), z], axis=1)
    return v * radius + np.asarray(center)


def icosphere(level: int = 4, radius: float = 1.0) -> np.ndarray:
    """Vertices of an icosahedron whose faces are split in four `level` times,
    projected on the sphere: 10·4^level + 2 points (2562 at level 4, the size
    of the paper's sphere cloud, §4.2)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
             (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
             (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts) * radius


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


@dataclasses.dataclass(frozen=True)
class Superquadric:
    """Superquadric solid F(p) <= 1 with F the usual inside-outside function.

    F(x, y, z) = (|x/a1|^(2/e2) + |y/a2|^(2/e2))^(e2/e1) + |z/a3|^(2/e1) in the
    body frame; world point p maps to the body frame by rot^T (p - center).
    """

    a: tuple
    e1: float
    e2: float
    center: tuple
    rot: tuple  # 3x3 row-major

    def body(self, p: np.ndarray) -> np.ndarray:
        return (p - np.asarray(self.center)) @ np.asarray(self.rot).reshape(3, 3)

    def F(self, p: np.ndarray) -> np.ndarray:
        b = self.body(p)
        a = np.asarray(self.a)
        ax = np.abs(b[:, 0] / a[0]) + 1e-300
        ay = np.abs(b[:, 1] / a[1]) + 1e-300
        az = np.abs(b[:, 2] / a[2]) + 1e-300
        return (ax ** (2 / self.e2) + ay ** (2 / self.e2)) ** (self.e2 / self.e1) + az ** (2 / self.e1)

    def sample_candidates(self, rng, m: int):
        """Surface points along random directions, with area weights.

        The solid is star-shaped about its centre and F is homogeneous of
        degree 2/e1, so the ray in direction w meets the surface at
        t = F(w)^(-e1/2). The surface area per unit solid angle is
        t^2 / |n . w| (n the unit normal), used as a rejection weight.
        """
        w = rng.normal(size=(m, 3))
        w /= np.linalg.norm(w, axis=1, keepdims=True)
        a = np.asarray(self.a)
        ax = np.abs(w[:, 0] / a[0]) + 1e-12
        ay = np.abs(w[:, 1] / a[1]) + 1e-12
        az = np.abs(w[:, 2] / a[2]) + 1e-12
        e1, e2 = self.e1, self.e2
        sxy = ax ** (2 / e2) + ay ** (2 / e2)
        Fw = sxy ** (e2 / e1) + az ** (2 / e1)
        t = Fw ** (-e1 / 2)
        pb = w * t[:, None]
        # gradient of F at the surface point (body frame), up to a positive factor
        bx = np.abs(pb[:, 0] / a[0]) + 1e-12
        by = np.abs(pb[:, 1] / a[1]) + 1e-12
        bz = np.abs(pb[:, 2] / a[2]) + 1e-12
        sxy_p = bx ** (2 / e2) + by ** (2 / e2)
        gx = (sxy_p ** (e2 / e1 - 1)) * bx ** (2 / e2 - 1) * np.sign(pb[:, 0]) / a[0] / e1
        gy = (sxy_p ** (e2 / e1 - 1)) * by ** (2 / e2 - 1) * np.sign(pb[:, 1]) / a[1] / e1
        gz = bz ** (2 / e1 - 1) * np.sign(pb[:, 2]) / a[2] / e1
        g = np.stack([gx, gy, gz], axis=1)
        gn = np.linalg.norm(g, axis=1) + 1e-300
        cosang = np.abs(np.sum(g * w, axis=1)) / gn
        weight = t * t / np.maximum(cosang, 1e-3)
        rot = np.asarray(self.rot).reshape(3, 3)
        p = pb @ rot.T + np.asarray(self.center)
        return p, weight


def random_superquadrics(rng, k: int = 3, fit_radius: float = 0.8):
    shapes = []
    for _ in range(k):
        a = rng.uniform(0.2, 0.35, 3)
        ext = float(np.linalg.norm(a))
        cdir = rng.normal(size=3)
        cdir /= np.linalg.norm(cdir)
        c = cdir * rng.uniform(0.0, max(0.0, fit_radius - ext))
        e1, e2 = rng.uniform(0.3, 3.0, 2)
        shapes.append(Superquadric(tuple(a), float(e1), float(e2), tuple(c), tuple(_random_rotation(rng).reshape(-1))))
    return shapes


def density_field(p: np.ndarray) -> np.ndarray:
    """Smooth sampling density 1 + 9 s(p), s in [0, 1]: a 10x variation."""
    s = 0.5 * (1.0 + np.sin(4.0 * p[:, 0] + 3.0 * p[:, 1] - 2.0 * p[:, 2]))
    return 1.0 + 9.0 * s


def superquadric_union_cloud(n: int = 1_000_000, k: int = 3, seed: int = 2, fit_radius: float = 0.8,
                             shapes=None) -> np.ndarray:
    """Points on the boundary of a union of k overlapping superquadrics.

    Candidates come from :meth:`Superquadric.sample_candidates`; a candidate
    is kept with probability proportional to (area weight, capped at 8x the
    median) x (density 1 + 9 s(p)), and only if it lies outside every other
    solid of the union. The kept points are shuffled and the first n returned.
    """
    rng = np.random.default_rng(seed)
    if shapes is None:
        shapes = random_superquadrics(rng, k, fit_radius)
    batches = []
    have = 0
    while have < n:
        m = max(200_000, (n - have) * 2)
        for i, s in enumerate(shapes):
            p, w = s.sample_candidates(rng, m)
            w = np.minimum(w, 8.0 * np.median(w))
            w = w * density_field(p)
            keep = rng.uniform(0.0, 1.0, m) * w.max() < w
            for j, o in enumerate(shapes):
                if j != i:
                    keep &= o.F(p) > 1.0
            batches.append(p[keep])
            have += int(keep.sum())
    pts = np.concatenate(batches)
    rng.shuffle(pts, axis=0)
    return np.ascontiguousarray(pts[:n])


# --------------------------------------------------------------------------
# Workload descriptions (sizes and seeds of the benchmarked configurations)
# --------------------------------------------------------------------------

def workload_circle64():
    """2-D, FP64, Q1: 200 noisy circle points, 64x64 grid on [-1,1]^2,
    u0 = circle of radius 0.9, 100 steps, full grid."""
    return dict(name="circle200_64sq_q1_fp64_full", grid=cube_grid(2, 64), cloud=circle_noisy(200, 0.5, 0.005, 0),
                u0_radius=0.9, interp=0, precision=64, band=0, steps=100)


def workload_torus128():
    """3-D torus, 20k points, 128^3 on [-1,1]^3, u0 = sphere r=0.9, band 6h."""
    return dict(name="torus20k_128cube_band6h", grid=cube_grid(3, 128), cloud=torus_cloud(20000, 0.5, 0.2, 0.002, 1),
                u0_radius=0.9, band=1)


def workload_superquadric256(n_points: int = 1_000_000):
    """3-D, 1M points on a union of 3 superquadrics (10x density variation),
    256^3 on [-1,1]^3, u0 = sphere r=0.9, band 6h."""
    return dict(name="sq3union1M_256cube_band6h", grid=cube_grid(3, 256),
                cloud=superquadric_union_cloud(n_points, 3, 2), u0_radius=0.9, band=1)


def batch_mix(seed: int = 3, n_jobs: int = 64, scale: float = 1.0):
    """Mixed batch: half 2-D (grids 64^2..512^2) and half 3-D (64^3..192^3),
    log-uniform point counts 1k..200k on random tori, spheres and superquadric
    unions, Q1/WENO mixed. ``scale`` < 1 shrinks point counts for tests."""
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n_jobs):
        dim = 2 if j < n_jobs // 2 else 3
        if dim == 2:
            n = int(round(math.exp(rng.uniform(math.log(64), math.log(512)))))
        else:
            n = int(round(math.exp(rng.uniform(math.log(64), math.log(192)))))
        npts = max(16, int(round(scale * math.exp(rng.uniform(math.log(1000), math.log(200000))))))
        kind = int(rng.integers(0, 3))
        s = int(rng.integers(0, 2**31 - 1))
        if dim == 2:
            if kind == 0:
                cloud = circle_noisy(npts, rng.uniform(0.3, 0.7), 0.003, s)
            elif kind == 1:
                c = circle_noisy(npts, 1.0, 0.0, s)
                cloud = c * np.array([rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7)])
            else:
                t = np.random.default_rng(s).uniform(0, 2 * np.pi, npts)
                r = 0.45 + 0.15 * np.cos(3 * t)
                cloud = np.stack([r * np.cos(t), r * np.sin(t)], axis=1)
        else:
            if kind == 0:
                cloud = torus_cloud(npts, rng.uniform(0.35, 0.55), rng.uniform(0.1, 0.2), 0.002, s)
            elif kind == 1:
                cloud = sphere_cloud(npts, rng.uniform(0.4, 0.75), 0.002, s)
            else:
                cloud = superquadric_union_cloud(npts, 3, s)
        jobs.append(dict(dim=dim, grid=cube_grid(dim, n), cloud=cloud, interp=int(rng.integers(0, 2)),
                         u0_radius=0.9, band=1, precision=32))
    return jobs
