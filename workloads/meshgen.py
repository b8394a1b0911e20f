"""Seeded synthetic tetrahedral meshes for the indentation workloads.

This module only builds inputs (node coordinates, tet connectivity, material ids
and fixed nodes). It holds none of the FEM arithmetic: no strain energy, no
stresses, no contact penalty. Both the CPU oracle and the CUDA path consume its
output.

Meshes:
  * ``cube_mesh``: unit cube, n x n x n hexes, each split into 6 tets (Kuhn split
    around the (0,0,0)->(1,1,1) diagonal; conforming because every hex uses the
    same split).
  * ``fingertip_mesh``: a two-layer half-capsule fingertip (a cylinder closed by
    one hemispherical cap, open at the base), built as a structured quad surface
    (cylinder grid + cubed-hemisphere cap with a matched seam) extruded inward
    along the surface normal into radial layers, each prism cut into 3 tets by
    the minimum-global-index diagonal rule so that shared quad faces are split
    the same way on both sides.

The paper meshes the BioTac skin with fTetWild (~4000 nodes, Sec. III-A); the
real geometry is not available, so these structured stand-ins are used instead.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SKIN, INNER = 0, 1


@dataclasses.dataclass
class Mesh:
    nodes: np.ndarray            # (Nn, 3) float64 reference coordinates
    tets: np.ndarray             # (Nt, 4) int32, positively oriented
    tet_material: np.ndarray     # (Nt,) int32 material id
    materials: np.ndarray        # (M, 2) float64 rows (E, nu)
    fixed_nodes: np.ndarray      # (Nf,) int32
    fixed_mask: np.ndarray | None = None   # (Nf,) uint8 bit0=x bit1=y bit2=z; None = all
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def _orient_positive(nodes: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Swap the last two vertices of every tet whose signed volume is negative."""
    x0 = nodes[tets[:, 0]]
    d1 = nodes[tets[:, 1]] - x0
    d2 = nodes[tets[:, 2]] - x0
    d3 = nodes[tets[:, 3]] - x0
    vol6 = np.einsum("ij,ij->i", d1, np.cross(d2, d3))
    tets = tets.copy()
    neg = vol6 < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    return tets


# ----------------------------------------------------------------------------- cube

def cube_mesh(n: int = 8, length: float = 1.0, E: float = 1.0e6, nu: float = 0.3,
              fix: str = "bottom") -> Mesh:
    """Unit cube of n^3 hexes, 6 tets each. ``fix``: 'bottom' (z=0 fully fixed),
    'rollers' (u_z=0 on z=0, u_x=0 on x=0, u_y=0 on y=0) or 'none'."""
    m = n + 1
    g = np.arange(m) * (length / n)
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    nodes = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)

    def nid(i, j, k):
        return i + m * (j + m * k)

    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                base = np.array([i, j, k])
                for p in perms:
                    c = base.copy()
                    verts = [nid(*c)]
                    for ax in p:
                        c[ax] += 1
                        verts.append(nid(*c))
                    tets.append(verts)
    tets = _orient_positive(nodes, np.asarray(tets, dtype=np.int64)).astype(np.int32)
    tet_material = np.zeros(len(tets), dtype=np.int32)
    materials = np.array([[E, nu]], dtype=np.float64)

    tol = 1e-12 * length
    if fix == "bottom":
        fixed = np.nonzero(nodes[:, 2] < tol)[0].astype(np.int32)
        mask = None
    elif fix == "rollers":
        bits = ((nodes[:, 0] < tol) * 1 + (nodes[:, 1] < tol) * 2
                + (nodes[:, 2] < tol) * 4).astype(np.uint8)
        fixed = np.nonzero(bits)[0].astype(np.int32)
        mask = bits[fixed]
    elif fix == "none":
        fixed = np.zeros(0, dtype=np.int32)
        mask = None
    else:
        raise ValueError(fix)
    return Mesh(nodes, tets, tet_material, materials, fixed, mask,
                name=f"cube{n}", meta={"n": n, "length": length})


# ------------------------------------------------------------------ fingertip

def _prism_to_tets(v):
    """Cut the prism (v0,v1,v2 | v3,v4,v5), v[i+3] above v[i], into 3 tets.

    Every quad face is split along the diagonal through its smallest global
    index, so two prisms sharing a quad face split it identically."""
    v = list(v)
    # rotate/reflect so that the globally smallest vertex is v[0]
    k = int(np.argmin(v))
    bottom, top = v[:3], v[3:]
    if k >= 3:
        bottom, top = top, bottom
        k -= 3
    bottom = bottom[k:] + bottom[:k]
    top = top[k:] + top[:k]
    a, b, c = bottom
    d, e, f = top
    if min(b, f) < min(c, e):
        return [(a, b, c, f), (a, b, f, e), (a, e, f, d)]
    return [(a, b, c, e), (a, e, c, f), (a, e, f, d)]


def _capsule_surface(R: float, Lc: float, n: int, m: int):
    """Quad surface of a capsule finger: cylinder (axis z, z in [0, Lc]) plus a
    hemispherical cap centred at (0, 0, Lc). Returns per surface node its foot
    point on the axis and its unit outward normal, plus the quads (index lists)."""
    assert n % 2 == 0 and n >= 2 and m >= 1
    nc = 4 * n                                   # nodes around the circumference
    theta = -math.pi / 4 + np.arange(nc) * (math.pi / 2 / n)
    foot, normal = [], []

    def add(f, nrm):
        idx = len(foot)
        foot.append(np.asarray(f, dtype=np.float64))
        normal.append(np.asarray(nrm, dtype=np.float64) / np.linalg.norm(nrm))
        return idx

    quads = []
    # cylinder rings z_l = Lc * l / m
    ring = np.empty((m + 1, nc), dtype=np.int64)
    for l in range(m + 1):
        z = Lc * l / m
        for j in range(nc):
            ring[l, j] = add((0.0, 0.0, z), (math.cos(theta[j]), math.sin(theta[j]), 0.0))
    for l in range(m):
        for j in range(nc):
            j1 = (j + 1) % nc
            quads.append((ring[l, j], ring[l, j1], ring[l + 1, j1], ring[l + 1, j]))

    # cubed hemisphere (equiangular): top face z=1 and upper halves of 4 sides.
    ang = -math.pi / 4 + np.arange(n + 1) * (math.pi / 2 / n)
    t = np.tan(ang)
    half = n // 2
    cap_foot = (0.0, 0.0, Lc)

    def face_grid(fn, ni, nj):
        grid = np.empty((ni, nj), dtype=np.int64)
        for i in range(ni):
            for j in range(nj):
                grid[i, j] = add(cap_foot, fn(i, j))
        return grid

    # side faces: azimuth block s covers theta in [-pi/4 + s*pi/2, pi/4 + s*pi/2];
    # local tangent u along increasing azimuth, height v from equator up.
    for s in range(4):
        c, sn = math.cos(s * math.pi / 2), math.sin(s * math.pi / 2)

        def fn(i, j, c=c, sn=sn):
            u, w = t[i], t[half + j]             # w in [0, 1]
            x, y = 1.0, u
            return (c * x - sn * y, sn * x + c * y, w)
        g = face_grid(fn, n + 1, half + 1)
        for i in range(n):
            for j in range(half):
                quads.append((g[i, j], g[i + 1, j], g[i + 1, j + 1], g[i, j + 1]))
    # top face
    g = face_grid(lambda i, j: (t[i], t[j], 1.0), n + 1, n + 1)
    for i in range(n):
        for j in range(n):
            quads.append((g[i, j], g[i + 1, j], g[i + 1, j + 1], g[i, j + 1]))
    foot, normal, quads = np.asarray(foot), np.asarray(normal), np.asarray(quads, dtype=np.int64)
    # merge coincident points (seam ring, cube edges) within a tolerance; the
    # first occurrence is kept, indices stay in order of first appearance.
    from scipy.spatial import cKDTree
    pos = foot + R * normal
    rep = np.arange(len(pos))
    for i, j in sorted(cKDTree(pos).query_pairs(1e-7 * R)):
        ri, rj = rep[i], rep[j]
        while rep[ri] != ri:
            ri = rep[ri]
        while rep[rj] != rj:
            rj = rep[rj]
        if ri != rj:
            rep[max(ri, rj)] = min(ri, rj)
    for i in range(len(rep)):
        r = i
        while rep[r] != r:
            r = rep[r]
        rep[i] = r
    keep = np.nonzero(rep == np.arange(len(rep)))[0]
    new_id = np.full(len(rep), -1, dtype=np.int64)
    new_id[keep] = np.arange(len(keep))
    return foot[keep], normal[keep], new_id[rep[quads]]


def fingertip_mesh(R: float = 7.0, L: float = 40.0, h: float = 0.88,
                   skin: float = 1.0, inner: float = 2.0,
                   E_skin: float = 1.5, nu_skin: float = 0.45,
                   E_inner: float = 0.2, nu_inner: float = 0.48,
                   n_skin: int | None = None, n_inner: int | None = None) -> Mesh:
    """Two-layer half-capsule fingertip in mm / MPa.

    Outer radius R, total length L (cylinder of length L-R plus a hemispherical
    cap), open at the base z=0. Radial layers: ``skin`` (material 0) over
    ``inner`` (material 1); the innermost node layer (radius R-skin-inner, the
    rigid core surface) is fully fixed."""
    Lc = L - R
    n = max(2, 2 * int(round(math.pi * R / (4.0 * h))))     # cap quads per cube edge (even)
    arc = (math.pi / 2) * R / n
    m = max(1, int(round(Lc / arc)))
    ns = n_skin if n_skin is not None else max(1, int(round(skin / h)))
    ni = n_inner if n_inner is not None else max(1, int(round(inner / h)))
    depths = np.concatenate([np.linspace(0.0, skin, ns + 1),
                             skin + np.linspace(0.0, inner, ni + 1)[1:]])
    foot, normal, quads = _capsule_surface(R, Lc, n, m)
    ns_nodes = len(foot)
    n_layers = len(depths)
    nodes = np.concatenate([foot + (R - d) * normal for d in depths], axis=0)

    # quads -> triangles, diagonal through the smallest surface index
    tris = []
    for q in quads:
        k = int(np.argmin(q))
        q = list(q[k:]) + list(q[:k])
        tris.append((q[0], q[1], q[2]))
        tris.append((q[0], q[2], q[3]))
    tets, mats = [], []
    for layer in range(n_layers - 1):
        mat = SKIN if layer < ns else INNER
        off_out, off_in = layer * ns_nodes, (layer + 1) * ns_nodes
        for a, b, c in tris:
            for tt in _prism_to_tets((a + off_in, b + off_in, c + off_in,
                                      a + off_out, b + off_out, c + off_out)):
                tets.append(tt)
                mats.append(mat)
    tets = _orient_positive(nodes, np.asarray(tets, dtype=np.int64)).astype(np.int32)
    fixed = np.arange((n_layers - 1) * ns_nodes, n_layers * ns_nodes, dtype=np.int32)
    materials = np.array([[E_skin, nu_skin], [E_inner, nu_inner]], dtype=np.float64)
    meta = {"R": R, "L": L, "Lc": Lc, "h": h, "n_cap": n, "m_axial": m,
            "n_skin": ns, "n_inner": ni, "n_surface": ns_nodes,
            "surface_foot": foot, "surface_normal": normal}
    return Mesh(nodes, tets, np.asarray(mats, dtype=np.int32), materials, fixed, None,
                name=f"fingertip_R{R:g}_h{h:.3g}", meta=meta)


def fingertip_tet_count(R: float, L: float, h: float, skin: float = 1.0,
                        inner: float = 2.0) -> int:
    """Tet count fingertip_mesh would produce, without building it."""
    Lc = L - R
    n = max(2, 2 * int(round(math.pi * R / (4.0 * h))))
    arc = (math.pi / 2) * R / n
    m = max(1, int(round(Lc / arc)))
    ns = max(1, int(round(skin / h)))
    ni = max(1, int(round(inner / h)))
    quads = 4 * n * m + n * n + 4 * n * (n // 2)
    return quads * 2 * 3 * (ns + ni)


def fingertip_for_tets(target: int, R: float, L: float = 40.0) -> float:
    """Pick h (by bisection on the log scale) so that the fingertip mesh has a
    tet count close to ``target``."""
    lo, hi = 0.05, 5.0
    best_h, best_err = hi, float("inf")
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        cnt = fingertip_tet_count(R, L, mid)
        err = abs(math.log(cnt / target))
        if err < best_err:
            best_h, best_err = mid, err
        if cnt > target:
            lo = mid
        else:
            hi = mid
    return best_h
