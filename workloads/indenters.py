"""Seeded rigid-indenter draws and their placement at initial contact.

An indenter is described exactly as the library's ``fem_set_indenter`` takes it:
shape id, pose (origin + 3x3 rotation, row-major), shape parameters, the unit
approach direction ``a`` and a depth schedule d_k measured along ``a`` from the
point of initial contact (Fig. 3 caption of the paper: indenter displacement is
relative to the point of initial contact).

Initial contact is found per candidate node as the first time at which the
indenter, translating along ``a``, reaches the node (ray-sphere, ray-cylinder,
slab tests); the earliest such time over all candidate nodes moves the pose to
the touching position. This is input preparation only; the contact penalty and
signed-distance arithmetic of the method live in the oracle and in the kernels.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SPHERE, CYLINDER, BOX, PLANE = 0, 1, 2, 3
SHAPE_NAMES = {SPHERE: "sphere", CYLINDER: "cylinder", BOX: "box", PLANE: "plane"}


@dataclasses.dataclass
class Indenter:
    shape: int
    origin: np.ndarray          # (3,)
    rotation: np.ndarray        # (3, 3), columns = local axes in world frame
    params: np.ndarray          # (3,) radius | radius | half extents | unused
    direction: np.ndarray       # (3,) unit approach direction a
    depth_schedule: np.ndarray  # (n_steps,) depths along a from initial contact

    @property
    def pose(self) -> np.ndarray:
        """origin(3) + rotation(9, row-major), the layout fem_set_indenter takes."""
        return np.concatenate([self.origin, self.rotation.reshape(-1)]).astype(np.float64)

    @property
    def n_steps(self) -> int:
        return int(len(self.depth_schedule))


def linear_schedule(depth: float, n_steps: int) -> np.ndarray:
    """d_k = depth * k / n_steps, k = 1..n_steps."""
    return depth * np.arange(1, n_steps + 1, dtype=np.float64) / n_steps


def _frame_from_axis(axis: np.ndarray) -> np.ndarray:
    """Rotation whose third column is ``axis`` (unit)."""
    z = axis / np.linalg.norm(axis)
    helper = np.array([1.0, 0.0, 0.0]) if abs(z[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    x = np.cross(helper, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z], axis=1)


def _perp_basis(a: np.ndarray):
    R = _frame_from_axis(a)
    return R[:, 0], R[:, 1]


def entry_times(ind: Indenter, X: np.ndarray) -> np.ndarray:
    """Time t at which each point X enters the indenter translated by t*a (the
    indenter moves, the point is still). +inf where the path misses it."""
    a = ind.direction
    c = ind.origin
    d = X - c
    t = np.full(len(X), np.inf)
    if ind.shape in (SPHERE, CYLINDER):
        r = ind.params[0]
        if ind.shape == CYLINDER:
            ax = ind.rotation[:, 2]
            d = d - np.outer(d @ ax, ax)
            aa = a - (a @ ax) * ax
        else:
            aa = a
        A = aa @ aa
        B = d @ aa
        C = np.einsum("ij,ij->i", d, d) - r * r
        disc = B * B - A * C
        ok = (disc >= 0) & (A > 0)
        t[ok] = (B[ok] - np.sqrt(disc[ok])) / A
    elif ind.shape == BOX:
        h = ind.params
        q = d @ ind.rotation          # local coords
        v = a @ ind.rotation
        lo = np.full(len(X), -np.inf)
        hi = np.full(len(X), np.inf)
        for k in range(3):
            if abs(v[k]) < 1e-15:
                miss = np.abs(q[:, k]) > h[k]
                lo[miss] = np.inf
                continue
            t1 = (q[:, k] - h[k]) / v[k]
            t2 = (q[:, k] + h[k]) / v[k]
            lo = np.maximum(lo, np.minimum(t1, t2))
            hi = np.minimum(hi, np.maximum(t1, t2))
        ok = lo <= hi
        t[ok] = lo[ok]
    elif ind.shape == PLANE:
        nrm = ind.rotation[:, 2]
        # half-space {y : (y - c) . nrm < 0}; X enters when (X - c - t a) . nrm = 0
        den = a @ nrm
        t = (d @ nrm) / den
    else:
        raise ValueError(ind.shape)
    return t


def place_at_contact(ind: Indenter, X: np.ndarray) -> Indenter:
    """Translate the indenter along a to the first touch of any point of X."""
    t = entry_times(ind, X)
    t0 = float(np.min(t))
    if not np.isfinite(t0):
        raise ValueError("indenter path misses every candidate node")
    return dataclasses.replace(ind, origin=ind.origin + t0 * ind.direction)


# ---------------------------------------------------------------- skin points

def sample_skin_point(rng: np.random.Generator, R: float, Lc: float, base_clear: float = 5.0):
    """Area-uniform point on the outer capsule surface, excluding the band within
    ``base_clear`` of the open base. Returns (point, outward normal)."""
    a_cyl = 2 * math.pi * R * (Lc - base_clear)
    a_cap = 2 * math.pi * R * R
    if rng.random() < a_cyl / (a_cyl + a_cap):
        th = rng.uniform(0.0, 2 * math.pi)
        z = rng.uniform(base_clear, Lc)
        nrm = np.array([math.cos(th), math.sin(th), 0.0])
        foot = np.array([0.0, 0.0, z])
    else:
        zc = rng.uniform(0.0, 1.0)          # uniform height => uniform area on a sphere
        ph = rng.uniform(0.0, 2 * math.pi)
        s = math.sqrt(max(0.0, 1 - zc * zc))
        nrm = np.array([s * math.cos(ph), s * math.sin(ph), zc])
        foot = np.array([0.0, 0.0, Lc])
    return foot + R * nrm, nrm


def _candidate_points(mesh) -> np.ndarray:
    """Outer-skin node positions (layer 0 of the fingertip generator)."""
    ns = mesh.meta["n_surface"]
    return mesh.nodes[:ns]


# -------------------------------------------------------------- workloads

def cube_sphere_indenter(radius: float = 0.3, depth: float = 0.05, n_steps: int = 10,
                         length: float = 1.0) -> Indenter:
    """Sphere centred over the top face of the unit cube, initial contact at the
    top-face centre node, approach direction -z."""
    c = np.array([0.5 * length, 0.5 * length, length + radius])
    return Indenter(SPHERE, c, np.eye(3), np.array([radius, 0.0, 0.0]),
                    np.array([0.0, 0.0, -1.0]), linear_schedule(depth, n_steps))


def cube_cylinder_indenter(radius: float = 0.3, depth: float = 0.05, n_steps: int = 10,
                           yaw_deg: float = 20.0, offset: float = 0.03) -> Indenter:
    """Infinite cylinder lying across the top face of the unit cube, axis
    horizontal (perpendicular to the approach -z) and turned ``yaw_deg`` from the
    x axis, line of contact shifted ``offset`` off the face centre; placed at
    initial contact with the top face and pressed along -z."""
    yaw = math.radians(yaw_deg)
    axis = np.array([math.cos(yaw), math.sin(yaw), 0.0])
    across = np.array([-math.sin(yaw), math.cos(yaw), 0.0])
    c = np.array([0.5, 0.5, 1.0 + radius]) + offset * across
    ind = Indenter(CYLINDER, c, _frame_from_axis(axis), np.array([radius, 0.0, 0.0]),
                   np.array([0.0, 0.0, -1.0]), linear_schedule(depth, n_steps))
    return ind


def cube_box_edge_indenter(half: float = 0.3, depth: float = 0.12, n_steps: int = 10,
                           yaw_deg: float = 15.0, offset: float = 0.03) -> Indenter:
    """Cube of half extent ``half`` presenting one edge to the top face of the
    unit cube: the edge is horizontal (turned ``yaw_deg`` from the x axis), the
    two faces meeting there lie at +-45 degrees to the approach -z, and the edge
    is shifted ``offset`` off the face centre. Nodes pressed under the edge fall
    on both sides of the box's medial plane through the edge."""
    yaw = math.radians(yaw_deg)
    edge = np.array([math.cos(yaw), math.sin(yaw), 0.0])
    a = np.array([0.0, 0.0, -1.0])
    w = np.cross(a, edge)
    rot = np.stack([(a + w) / math.sqrt(2.0), (a - w) / math.sqrt(2.0), edge], axis=1)
    across = np.array([-math.sin(yaw), math.cos(yaw), 0.0])
    centre = np.array([0.5, 0.5, 1.0 + half * math.sqrt(2.0)]) + offset * across
    return Indenter(BOX, centre, rot, np.array([half, half, half]), a, linear_schedule(depth, n_steps))


def plane_indenter(height: float, depth: float, n_steps: int) -> Indenter:
    """Rigid plane whose face sits at z=height, outward normal -z, pushed along -z."""
    R = np.array([[1.0, 0, 0], [0, -1.0, 0], [0, 0, -1.0]])   # third column = -z
    return Indenter(PLANE, np.array([0.0, 0.0, height]), R, np.zeros(3),
                    np.array([0.0, 0.0, -1.0]), linear_schedule(depth, n_steps))


def fingertip_sphere_indentation(mesh, seed: int = 1001, radius: float = 4.0,
                                 depth: float = 2.0, n_steps: int = 20) -> Indenter:
    """Sphere of radius r pressed normal to a seeded random skin point."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p, nrm = sample_skin_point(rng, mesh.meta["R"], mesh.meta["Lc"])
    ind = Indenter(SPHERE, p + radius * nrm, np.eye(3), np.array([radius, 0.0, 0.0]),
                   -nrm, linear_schedule(depth, n_steps))
    return place_at_contact(ind, _candidate_points(mesh))


def draw_indentation(mesh, rng: np.random.Generator, n_steps: int = 20) -> Indenter:
    """One random indentation: shape uniform over {sphere r~U[2,6], cylinder
    r~U[1,4] with a random axis normal to the approach, 20 mm cube presenting an
    edge}; skin point area-uniform; approach tilted by theta~U[0,30 deg] from the
    inward normal; depth~U[0.5, 3]."""
    shape = int(rng.integers(0, 3))
    p, nrm = sample_skin_point(rng, mesh.meta["R"], mesh.meta["Lc"])
    theta = math.radians(rng.uniform(0.0, 30.0))
    phi = rng.uniform(0.0, 2 * math.pi)
    t1, t2 = _perp_basis(nrm)
    out = math.cos(theta) * nrm + math.sin(theta) * (math.cos(phi) * t1 + math.sin(phi) * t2)
    a = -out / np.linalg.norm(out)
    depth = rng.uniform(0.5, 3.0)
    e1, e2 = _perp_basis(a)
    if shape == SPHERE:
        r = rng.uniform(2.0, 6.0)
        ind = Indenter(SPHERE, p - (r + 1.0) * a, np.eye(3), np.array([r, 0.0, 0.0]),
                       a, linear_schedule(depth, n_steps))
    elif shape == CYLINDER:
        r = rng.uniform(1.0, 4.0)
        psi = rng.uniform(0.0, math.pi)
        axis = math.cos(psi) * e1 + math.sin(psi) * e2
        ind = Indenter(CYLINDER, p - (r + 1.0) * a, _frame_from_axis(axis),
                       np.array([r, 0.0, 0.0]), a, linear_schedule(depth, n_steps))
    else:
        side = 20.0
        hh = side / 2
        psi = rng.uniform(0.0, 2 * math.pi)
        edge = math.cos(psi) * e1 + math.sin(psi) * e2
        w = np.cross(a, edge)
        rx = (a + w) / math.sqrt(2.0)
        ry = (a - w) / math.sqrt(2.0)
        rot = np.stack([rx, ry, edge], axis=1)
        centre = p - (hh * math.sqrt(2.0) + 1.0) * a
        ind = Indenter(BOX, centre, rot, np.array([hh, hh, hh]), a,
                       linear_schedule(depth, n_steps))
    return place_at_contact(ind, _candidate_points(mesh))


def draw_indentations(mesh, n: int, seed: int, n_steps: int = 20):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [draw_indentation(mesh, rng, n_steps) for _ in range(n)]
