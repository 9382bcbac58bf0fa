"""Seeded synthetic scenes for the Embedded-IPC contact stage.

This module only builds inputs: surface meshes, the tetrahedral cage, the barycentric
embedding weights (the set-up step of Sec. III-D, computed once at t = 0), the kinematic
positions and the reduced-coordinate iterates q along a prescribed motion.  It holds none
of the contact-stage arithmetic (distances, barrier, friction, derivatives, CCD): both the
CUDA library and the CPU oracle receive the arrays built here and compute everything else
on their own.

Layout of a `Scene` (all numpy, C-contiguous):
  tris     int32 [F,3]   surface triangles of every body, vertex ids into [0, Nv)
  edges    int32 [E,2]   unique undirected edges (a < b), sorted lexicographically
  cage_idx int32 [Nv,4]  cage-node ids of the containing tet (Sec. III-D, i^j(k)); -1 row
                         for a kinematic vertex (prescribed, no reduced DoF)
  w        f64   [Nv,4]  barycentric weights omega^k_j of Eq. 13-14
  x_kin    f64   [Nv,3]  positions of kinematic vertices (zero rows for embedded ones)
  Ns       number of cage nodes; q has shape [Ns,3]
  body     int32 [Nv]    body id of each vertex (informational)

Paper workloads are replaced by these stand-ins (the paper's meshes and recorded
trajectories are not public): an icosphere on a rigid pad (small latency case), a noisy
sphere squeezed by two ellipsoidal membranes (bubble-gripper grasp, Sec. IV-A) and a thin
plate lowered between rigid tines (dish rack, Sec. IV-B).
"""
from __future__ import annotations

import dataclasses
import functools
import math
from typing import Callable, Dict, List, Tuple

import numpy as np

# Contact parameters of Sec. IV-A: kappa = 1e4, dhat = 1e-3 m, eps_v = 1e-3 m/s; the time
# step h = 0.01 s is the middle of the three step sizes of the convergence study.
DEFAULT_PARAMS = dict(dhat=1e-3, kappa=1e4, mu=0.5, eps_v=1e-3, h=1e-2,
                      accd_s=0.1, accd_max_iter=10000)


@dataclasses.dataclass
class Scene:
    name: str
    tris: np.ndarray
    edges: np.ndarray
    cage_idx: np.ndarray
    w: np.ndarray
    x_kin: np.ndarray
    Ns: int
    cage_tets: np.ndarray
    q_rest: np.ndarray
    body: np.ndarray
    params: Dict[str, float]
    # iterate(t) -> q [Ns,3]; lag_of(t) -> iterate index whose state lags friction;
    # dq(t) -> [Ns,3] search direction handed to the CCD step bound.
    n_iterates: int = 1
    iterate: Callable[[int], np.ndarray] = None
    lag_of: Callable[[int], int] = None
    dq: Callable[[int], np.ndarray] = None

    @property
    def Nv(self) -> int:
        return int(self.cage_idx.shape[0])

    @property
    def F(self) -> int:
        return int(self.tris.shape[0])

    @property
    def E(self) -> int:
        return int(self.edges.shape[0])

    @property
    def kinematic(self) -> np.ndarray:
        return self.cage_idx[:, 0] < 0


# ----------------------------------------------------------------------------- meshes

def _icosahedron() -> Tuple[np.ndarray, np.ndarray]:
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
                  (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)],
                 dtype=np.float64)
    f = np.array([(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9),
                  (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2),
                  (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
                  (8, 6, 7), (9, 8, 1)], dtype=np.int64)
    return v / np.linalg.norm(v, axis=1, keepdims=True), f


def icosphere(level: int) -> Tuple[np.ndarray, np.ndarray]:
    """Unit icosphere by recursive edge-midpoint subdivision (10*4^L+2 verts, 20*4^L tris)."""
    v, f = _icosahedron()
    verts = [tuple(p) for p in v]
    faces = [tuple(x) for x in f]
    for _ in range(level):
        cache: Dict[Tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                p = (np.array(verts[a]) + np.array(verts[b])) * 0.5
                p /= np.linalg.norm(p)
                cache[key] = len(verts)
                verts.append(tuple(p))
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts, dtype=np.float64), np.array(faces, dtype=np.int32)


def geodesic_sphere(n: int) -> Tuple[np.ndarray, np.ndarray]:
    """Unit geodesic sphere of frequency n: each icosahedron face cut into n^2 triangles,
    points projected to the sphere (10 n^2 + 2 verts, 20 n^2 tris)."""
    v, f = _geodesic_sphere_cached(int(n))
    return v.copy(), f.copy()


@functools.lru_cache(maxsize=None)
def _geodesic_sphere_cached(n: int) -> Tuple[np.ndarray, np.ndarray]:
    base_v, base_f = _icosahedron()
    index: Dict[tuple, int] = {}
    pts: List[np.ndarray] = []
    tris: List[Tuple[int, int, int]] = []

    def vid(a, b, c, wa, wb, wc) -> int:
        key = tuple(sorted((x, wx) for x, wx in ((a, wa), (b, wb), (c, wc)) if wx > 0))
        k = index.get(key)
        if k is None:
            p = (wa * base_v[a] + wb * base_v[b] + wc * base_v[c]) / n
            p = p / np.linalg.norm(p)
            k = len(pts)
            index[key] = k
            pts.append(p)
        return k

    for a, b, c in base_f:
        grid = {}
        for i in range(n + 1):
            for j in range(n + 1 - i):
                grid[(i, j)] = vid(a, b, c, n - i - j, i, j)
        for i in range(n):
            for j in range(n - i):
                tris.append((grid[(i, j)], grid[(i + 1, j)], grid[(i, j + 1)]))
                if i + j < n - 1:
                    tris.append((grid[(i + 1, j)], grid[(i + 1, j + 1)], grid[(i, j + 1)]))
    return np.array(pts, dtype=np.float64), np.array(tris, dtype=np.int32)


def grid_plane(nx: int, ny: int, x0: float, x1: float, y0: float, y1: float):
    """Triangulated rectangle in the z = 0 plane with nx*ny cells (2 tris each)."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    v = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    idx = np.arange((nx + 1) * (ny + 1)).reshape(nx + 1, ny + 1)
    a = idx[:-1, :-1].ravel(); b = idx[1:, :-1].ravel()
    c = idx[1:, 1:].ravel(); d = idx[:-1, 1:].ravel()
    f = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)])
    return v, f.astype(np.int32)


def box_surface(lx: float, ly: float, lz: float, nx: int, ny: int, nz: int):
    """Closed triangulated box [-lx/2,lx/2]x[-ly/2,ly/2]x[-lz/2,lz/2] with a structured
    grid of nx x ny x nz cells per direction on its faces (shared boundary vertices)."""
    xs = np.linspace(-lx / 2, lx / 2, nx + 1)
    ys = np.linspace(-ly / 2, ly / 2, ny + 1)
    zs = np.linspace(-lz / 2, lz / 2, nz + 1)
    index: Dict[Tuple[int, int, int], int] = {}
    pts: List[Tuple[float, float, float]] = []

    def vid(i, j, k):
        key = (i, j, k)
        if key not in index:
            index[key] = len(pts)
            pts.append((xs[i], ys[j], zs[k]))
        return index[key]

    tris: List[Tuple[int, int, int]] = []

    def quad_face(fixed_axis, fixed_val, n1, n2, flip):
        for u in range(n1):
            for v in range(n2):
                def P(a, b):
                    ijk = [0, 0, 0]
                    o = [ax for ax in range(3) if ax != fixed_axis]
                    ijk[fixed_axis] = fixed_val
                    ijk[o[0]] = a
                    ijk[o[1]] = b
                    return vid(*ijk)
                p00, p10, p11, p01 = P(u, v), P(u + 1, v), P(u + 1, v + 1), P(u, v + 1)
                if flip:
                    tris.extend([(p00, p11, p10), (p00, p01, p11)])
                else:
                    tris.extend([(p00, p10, p11), (p00, p11, p01)])

    quad_face(0, 0, ny, nz, True); quad_face(0, nx, ny, nz, False)
    quad_face(1, 0, nx, nz, False); quad_face(1, ny, nx, nz, True)
    quad_face(2, 0, nx, ny, True); quad_face(2, nz, nx, ny, False)
    return np.array(pts, dtype=np.float64), np.array(tris, dtype=np.int32)


def open_cylinder(radius: float, height: float, n_around: int, n_up: int):
    """Open tube along z from 0 to height: n_around segments, n_up rings of quads."""
    th = 2 * np.pi * np.arange(n_around) / n_around
    zs = np.linspace(0.0, height, n_up + 1)
    v = np.array([(radius * math.cos(t), radius * math.sin(t), z) for z in zs for t in th])
    tris = []
    for r in range(n_up):
        for s in range(n_around):
            a = r * n_around + s
            b = r * n_around + (s + 1) % n_around
            c = (r + 1) * n_around + (s + 1) % n_around
            d = (r + 1) * n_around + s
            tris += [(a, b, c), (a, c, d)]
    return v, np.array(tris, dtype=np.int32)


def edges_of(tris: np.ndarray) -> np.ndarray:
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]).astype(np.int64)
    e.sort(axis=1)
    # unique rows in lexicographic order, via one int64 key per row
    n = int(e.max()) + 1 if len(e) else 1
    key = np.sort(e[:, 0] * n + e[:, 1])
    key = key[np.concatenate([[True], key[1:] != key[:-1]])] if len(key) else key
    e = np.stack([key // n, key % n], 1)
    return np.ascontiguousarray(e.astype(np.int32))


# ----------------------------------------------------------------------------- cages

def grid_cage(lo, hi, dims):
    """Regular node grid over the box [lo,hi] with dims = (nx,ny,nz) cubes, each split into
    five tets; the split alternates with (i+j+k) mod 2 so shared faces conform."""
    nx, ny, nz = dims
    lo = np.asarray(lo, float); hi = np.asarray(hi, float)
    xs = np.linspace(lo[0], hi[0], nx + 1)
    ys = np.linspace(lo[1], hi[1], ny + 1)
    zs = np.linspace(lo[2], hi[2], nz + 1)
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    nodes = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)

    def nid(i, j, k):
        return (i * (ny + 1) + j) * (nz + 1) + k

    even = [(0, 4, 2, 1), (6, 2, 4, 7), (5, 4, 1, 7), (3, 1, 2, 7), (4, 2, 1, 7)]
    odd = [(4, 0, 5, 6), (2, 0, 6, 3), (1, 0, 3, 5), (7, 5, 3, 6), (0, 6, 5, 3)]
    tets = []
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                c = [nid(i + (b >> 2 & 1), j + (b >> 1 & 1), k + (b & 1)) for b in range(8)]
                for t in (even if (i + j + k) % 2 == 0 else odd):
                    tets.append([c[t[0]], c[t[1]], c[t[2]], c[t[3]]])
    tets = np.array(tets, dtype=np.int64)
    # orient every tet positively
    p = nodes[tets]
    vol = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    flip = vol < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    return nodes, tets.astype(np.int32), (lo, hi, np.array(dims))


def embed_weights(points: np.ndarray, nodes: np.ndarray, tets: np.ndarray, grid) -> Tuple[np.ndarray, np.ndarray]:
    """Containing tet and barycentric weights of each point (Sec. III-D, set-up at t=0).

    The tet chosen is the lowest-index tet whose four barycentrics are all >= -1e-12; the
    grid lets us test only the five tets of each of the (up to 8) cubes a point touches."""
    lo, hi, dims = grid
    h = (hi - lo) / dims
    nyz = dims[1] * dims[2]
    best_t = np.full(len(points), np.iinfo(np.int64).max, dtype=np.int64)
    best_w = np.zeros((len(points), 4))
    rel = (points - lo) / h
    base = np.floor(rel).astype(np.int64)
    # A point more than 1e-8 cells inside its own cube has barycentrics below -1e-9 in every
    # tet of the other cubes, so only points near a cube face search the 26 neighbours.
    fr = rel - base
    near = np.nonzero(np.any((fr < 1e-8) | (fr > 1.0 - 1e-8), axis=1))[0]
    everyone = np.arange(len(points))
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for dk in (-1, 0, 1):
                cand = near if (di or dj or dk) else everyone
                cell = base[cand] + np.array([di, dj, dk])
                inside = np.all((cell >= 0) & (cell < dims), axis=1)
                sel, cell = cand[inside], cell[inside]
                if len(sel) == 0:
                    continue
                cid = cell[:, 0] * nyz + cell[:, 1] * dims[2] + cell[:, 2]
                for s in range(5):
                    t = cid * 5 + s
                    v = nodes[tets[t]]
                    D = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
                    lam = np.linalg.solve(D, (points[sel] - v[:, 0])[:, :, None])[:, :, 0]
                    wts = np.concatenate([1.0 - lam.sum(1, keepdims=True), lam], 1)
                    good = np.all(wts >= -1e-12, axis=1) & (t < best_t[sel])
                    best_t[sel[good]] = t[good]
                    best_w[sel[good]] = wts[good]
    if np.any(best_t == np.iinfo(np.int64).max):
        raise ValueError("point outside the cage")
    return tets[best_t].astype(np.int32), best_w


# ----------------------------------------------------------------------------- noise

class GradientNoise:
    """Seeded lattice gradient noise (Perlin-style): random unit gradients on the integer
    lattice, quintic fade, trilinear blend of the corner dot products."""

    def __init__(self, seed: int, size: int = 256):
        rng = np.random.default_rng(seed)
        g = rng.normal(size=(size, 3))
        self.grad = g / np.linalg.norm(g, axis=1, keepdims=True)
        self.perm = rng.permutation(size)
        self.size = size

    def _hash(self, i, j, k):
        s = self.size
        return self.perm[(self.perm[(self.perm[i % s] + j) % s] + k) % s]

    def __call__(self, p: np.ndarray) -> np.ndarray:
        i0 = np.floor(p).astype(np.int64)
        f = p - i0
        u = f * f * f * (f * (f * 6 - 15) + 10)
        out = np.zeros(len(p))
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    g = self.grad[self._hash(i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz)]
                    d = f - np.array([dx, dy, dz])
                    wgt = ((u[:, 0] if dx else 1 - u[:, 0]) * (u[:, 1] if dy else 1 - u[:, 1])
                           * (u[:, 2] if dz else 1 - u[:, 2]))
                    out += wgt * np.einsum("ij,ij->i", g, d)
        return out


def fractal_noise(p: np.ndarray, seed: int, octaves: int = 3, freq: float = 2.0) -> np.ndarray:
    n = GradientNoise(seed)
    out = np.zeros(len(p)); amp = 1.0
    for o in range(octaves):
        out += amp * n(p * freq * (2 ** o) + 17.0 * o)
        amp *= 0.5
    return out / np.max(np.abs(out))


# ----------------------------------------------------------------------------- assembly

class _Builder:
    """Concatenates bodies: embedded bodies own a block of cage nodes, kinematic bodies own
    none."""

    def __init__(self):
        self.verts, self.tris, self.cage_idx, self.w, self.kin, self.body = [], [], [], [], [], []
        self.nodes, self.tets = [], []
        self.nv = 0
        self.ns = 0
        self.nbody = 0

    def add_embedded(self, verts, tris, nodes, tets, grid):
        idx, w = embed_weights(verts, nodes, tets, grid)
        node_off = self.ns
        self._add(verts, tris, idx + node_off, w, np.zeros_like(verts))
        self.nodes.append(nodes)
        self.tets.append(tets + node_off)
        self.ns += len(nodes)
        return slice(node_off, node_off + len(nodes))

    def add_kinematic(self, verts, tris):
        self._add(verts, tris, np.full((len(verts), 4), -1, np.int32), np.zeros((len(verts), 4)), verts)

    def _add(self, verts, tris, idx, w, xk):
        self.tris.append(tris + self.nv)
        self.cage_idx.append(idx.astype(np.int32))
        self.w.append(w)
        self.kin.append(xk)
        self.body.append(np.full(len(verts), self.nbody, np.int32))
        self.nbody += 1
        self.nv += len(verts)

    def scene(self, name, params) -> Scene:
        tris = np.ascontiguousarray(np.concatenate(self.tris).astype(np.int32))
        return Scene(name=name, tris=tris, edges=edges_of(tris),
                     cage_idx=np.ascontiguousarray(np.concatenate(self.cage_idx)),
                     w=np.ascontiguousarray(np.concatenate(self.w)),
                     x_kin=np.ascontiguousarray(np.concatenate(self.kin)),
                     Ns=self.ns, cage_tets=np.concatenate(self.tets) if self.tets else np.zeros((0, 4), np.int32),
                     q_rest=np.ascontiguousarray(np.concatenate(self.nodes)) if self.nodes else np.zeros((0, 3)),
                     body=np.concatenate(self.body), params=dict(params))


def embedded_positions(scene: Scene, q: np.ndarray) -> np.ndarray:
    """Positions used only to place bodies while building a scene."""
    x = np.einsum("vj,vjk->vk", scene.w, q[np.maximum(scene.cage_idx, 0)])
    kin = scene.kinematic
    x[kin] = scene.x_kin[kin]
    return x


def sphere_on_pad(seed: int = 0, level: int = 4, pad_cells: int = 64, cage_cubes: int = 6,
                  radius: float = 0.05, gap_frac: float = 0.3) -> Scene:
    """Level-4 icosphere (r = 5 cm) embedded in a 6^3-cube, 5-tet cage (343 nodes) resting
    0.3 dhat above a kinematic 64x64-cell pad at z = 0.  Cage nodes get N(0, 1 mm)
    jitter; the iterate list is [q0, q0 + alpha/2 dq] where alpha is supplied by the caller
    (see `with_second_iterate`)."""
    params = dict(DEFAULT_PARAMS)
    dhat = params["dhat"]
    rng = np.random.default_rng(seed)
    sv, st = icosphere(level)
    sv = sv * radius
    half = radius * 1.2
    nodes, tets, grid = grid_cage([-half] * 3, [half] * 3, (cage_cubes,) * 3)
    pv, pt = grid_plane(pad_cells, pad_cells, -0.1, 0.1, -0.1, 0.1)
    b = _Builder()
    b.add_embedded(sv, st, nodes, tets, grid)
    b.add_kinematic(pv, pt)
    sc = b.scene("sphere_on_pad", params)
    q = sc.q_rest + rng.normal(0.0, 1e-3, size=sc.q_rest.shape)
    x = embedded_positions(sc, q)
    zmin = x[~sc.kinematic, 2].min()
    q[:, 2] += gap_frac * dhat - zmin
    dq_raw = 0.5 * rng.normal(size=q.shape) + np.array([0.0, 0.0, -1.0])
    sc_tmp = dataclasses.replace(sc)
    dx = embedded_positions(sc_tmp, dq_raw)
    dx[sc.kinematic] = 0.0
    dq = dq_raw * (5e-3 / np.linalg.norm(dx, axis=1).max())
    q0 = q.copy()
    sc.n_iterates = 1
    sc.iterate = lambda t: q0.copy()
    sc.lag_of = lambda t: 0
    sc.dq = lambda t: dq.copy()
    return sc


def with_second_iterate(sc: Scene, alpha: float) -> Scene:
    """Adds the iterate q0 + alpha/2 dq (friction then sees u != 0)."""
    q0 = sc.iterate(0)
    dq = sc.dq(0)
    q1 = q0 + 0.5 * alpha * dq
    out = dataclasses.replace(sc)
    out.n_iterates = 2
    out.iterate = lambda t: (q0 if t == 0 else q1).copy()
    out.lag_of = lambda t: 0
    return out


def _ellipsoid(n: int, axes) -> Tuple[np.ndarray, np.ndarray]:
    v, f = geodesic_sphere(n)
    # put an icosahedron vertex on the -y pole: rotate base vertex 0 (which is (-1,t,0)/|.|)
    a = v[0] / np.linalg.norm(v[0])
    target = np.array([0.0, -1.0, 0.0])
    axis = np.cross(a, target); s = np.linalg.norm(axis); c = float(a @ target)
    if s > 1e-15:
        k = axis / s
        K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        R = np.eye(3) + s * K + (1 - c) * K @ K
        v = v @ R.T
    return v * np.asarray(axes), f


def bubble_grasp(seed: int = 0, n_body: int = 71, n_mem: int = 45,
                 body_cage=(10, 11, 11), mem_cage=(19, 5, 16), n_steps: int = 20,
                 iters_per_step: int = 3, closing_per_step: float = 1e-3) -> Scene:
    """Noisy sphere (R = 5 cm, 5% radial gradient noise, geodesic frequency n_body) in a
    ~1.5k-node cage, squeezed along y by two ellipsoidal membranes (semi-axes 6 x 1.5 x 4 cm,
    frequency n_mem) each in a ~2k-node cage.  dhat = 5e-4 m, mu = 0.8.

    Motion (kinematic replay, n_steps x iters_per_step iterates): the body cage is scaled
    in y about the body centre so that its highest point moves in by `closing_per_step` per
    step, the membranes translate to keep a gap g(t) in [0.2, 0.8] dhat above the body's
    extreme y, and they flatten slightly.  Every iterate, and every straight path between
    consecutive iterates, keeps the bodies on opposite sides of the planes y = +-(ymax +
    g/2), so the trajectory is intersection-free by construction.  The CCD direction dq(t)
    is the motion to the next iterate plus a push of the membranes by 1.5 gaps toward the
    body, so that the step bound is active."""
    params = dict(DEFAULT_PARAMS, dhat=5e-4, mu=0.8)
    dhat = params["dhat"]
    R = 0.05
    rng = np.random.default_rng(seed)
    bv, bt = geodesic_sphere(n_body)
    noise = fractal_noise(bv * 1.0, seed=seed + 101)
    bv = bv * (R * (1.0 + 0.05 * noise))[:, None]
    ext = np.abs(bv).max(0) + 2e-3
    bn, btet, bgrid = grid_cage(-ext, ext, body_cage)
    axes = np.array([0.06, 0.015, 0.04])
    mv, mt = _ellipsoid(n_mem, axes)
    mext = axes + 1.5e-3
    mn, mtet, mgrid = grid_cage(-mext, mext, mem_cage)
    b = _Builder()
    sl_body = b.add_embedded(bv, bt, bn, btet, bgrid)
    # membrane at -y: pole vertex (0,-b,0) is its innermost point for the +y membrane; place
    # the +y membrane with that pole facing the body, and mirror for the -y one.
    mv_top = mv.copy()                                  # pole at -y, faces the body from +y
    mv_bot = mv.copy() * np.array([1.0, -1.0, 1.0])     # pole at +y
    mt_bot = mt[:, [0, 2, 1]]
    sl_top = b.add_embedded(mv_top, mt, mn, mtet, mgrid)
    sl_bot = b.add_embedded(mv_bot, mt_bot, mn, mtet, mgrid)   # the cage box is symmetric
    sc = b.scene("bubble_grasp", params)
    body_rest = sc.q_rest[sl_body].copy()
    ymax0 = bv[:, 1].max()
    ymin0 = bv[:, 1].min()
    yc = 0.5 * (ymax0 + ymin0)
    n_it = n_steps * iters_per_step
    # seeded gap schedule in [0.2, 0.8] dhat, smooth in t
    ph = rng.uniform(0, 2 * np.pi, size=3)
    ts = np.arange(n_it + 2)
    gap = dhat * (0.5 + 0.3 * np.sin(2 * np.pi * ts / 23.0 + ph[0]) * np.cos(2 * np.pi * ts / 41.0 + ph[1]))
    # per-node smooth wobble of the body cage in x/z (tangential motion for friction)
    wob = rng.normal(size=(3,)) * 2e-4
    mem_top_rest = sc.q_rest[sl_top].copy()
    mem_bot_rest = sc.q_rest[sl_bot].copy()

    def q_at(t: float) -> np.ndarray:
        closing = closing_per_step * t / iters_per_step
        half_up = ymax0 - yc
        half_dn = yc - ymin0
        s_up = (half_up - closing) / half_up
        s_dn = (half_dn - closing) / half_dn
        q = sc.q_rest.copy()
        qb = body_rest.copy()
        rel = qb[:, 1] - yc
        qb[:, 1] = yc + np.where(rel >= 0, rel * s_up, rel * s_dn)
        qb[:, 0] += wob[0] * t * (qb[:, 2] / R)
        qb[:, 2] += wob[2] * t * (qb[:, 0] / R)
        q[sl_body] = qb
        ti = int(math.floor(t)); fr = t - ti
        g = (1 - fr) * gap[ti] + fr * gap[ti + 1]
        flat = 1.0 - 0.1 * t / n_it            # membranes flatten by up to 10% in y
        mt_ = mem_top_rest.copy()
        mt_[:, 1] = mt_[:, 1] * flat
        mt_[:, 1] += (yc + half_up * s_up) + g + axes[1] * flat
        q[sl_top] = mt_
        mb_ = mem_bot_rest.copy()
        mb_[:, 1] = mb_[:, 1] * flat
        mb_[:, 1] -= (half_dn * s_dn - yc) + g + axes[1] * flat
        q[sl_bot] = mb_
        return q

    def dq_at(t: int) -> np.ndarray:
        # next-iterate motion plus a push of both membranes toward the body by 1.5 gaps,
        # so the step bound cuts the step at about two thirds
        d = q_at(float(t) + 1.0) - q_at(float(t))
        d[sl_top, 1] -= 1.5 * gap[t]
        d[sl_bot, 1] += 1.5 * gap[t]
        return d

    sc.n_iterates = n_it
    sc.iterate = lambda t: q_at(float(t))
    sc.lag_of = lambda t: (t // iters_per_step) * iters_per_step
    sc.dq = dq_at
    sc.node_slices = dict(body=sl_body, top=sl_top, bottom=sl_bot)
    return sc


def bubble_grasp_physical(seed: int = 0, small: bool = False, n_steps: int = 10, closing: float = 1e-4) -> Scene:
    """The bubble-grasp geometry simulated instead of replayed (Sec. IV-A set-up): the body
    (E = 5e4 Pa, nu = 0.45, rho = 1e3 kg/m^3) and both membranes (E = 1e4 Pa, nu = 0.45,
    rho = 10 kg/m^3) are elastic cages under gravity; each membrane's outermost cage layer
    (away from the body) is position-controlled, moving toward the body by `closing` per
    time step (h = 1e-2 s); everything else is free.  Friction lags once per time step.
    Inputs for the driver: q0, prescribed_nodes, prescribed_q(n), materials, gravity."""
    if small:
        sc = bubble_grasp(seed, n_body=16, n_mem=10, body_cage=(5, 5, 5), mem_cage=(8, 3, 6))
    else:
        sc = bubble_grasp(seed)
    sc.name = "bubble_grasp_physical" + ("_small" if small else "")
    q0 = sc.iterate(0)
    sc.q0 = q0
    presc = np.zeros(sc.Ns, bool)
    sign = np.zeros(sc.Ns)
    for name, sgn in (("top", -1.0), ("bottom", 1.0)):
        sl = sc.node_slices[name]
        y = q0[sl, 1]
        layer = np.abs(y - (y.max() if sgn < 0 else y.min())) < 1e-9
        idx = np.arange(sc.Ns)[sl][layer]
        presc[idx] = True
        sign[idx] = sgn
    sc.prescribed_nodes = presc
    sc.fixed_nodes = presc
    sc.prescribed_q = lambda n: q0 + (n * closing * sign)[:, None] * np.array([0.0, 1.0, 0.0])
    sc.materials = {0: dict(E=5e4, nu=0.45, rho=1e3), 1: dict(E=1e4, nu=0.45, rho=10.0),
                    2: dict(E=1e4, nu=0.45, rho=10.0)}
    sc.gravity = np.array([0.0, 0.0, -9.81])
    sc.n_steps = int(n_steps)
    sc.lag_every_step = True
    return sc


def plate_in_rack(seed: int = 0, plate_cells=(150, 100), n_tines: int = 10,
                  tine_segs=(40, 50), plate_cage=(19, 1, 19), n_iters: int = 100,
                  lower_per_iter: float = 5e-4) -> Scene:
    """Thin plate (20 x 15 cm, 2 mm thick, ~60k tris, in a 20x2x20-node cage) lowered
    0.5 mm per iteration between two rows of rigid open tubes (r = 3 mm, 15 cm tall,
    40 x 50 quads each, 25 mm pitch, kinematic).  The plate is tilted ~2 degrees in its
    own plane so its grid edges run nearly parallel to the tube generators.  The tube
    walls facing the plate sit 0.5 dhat from the plate faces; the plate stays inside
    |y| <= 1 mm and the tubes outside it, so the motion is intersection-free.
    dhat = 2e-4 m, mu = 0.5."""
    params = dict(DEFAULT_PARAMS, dhat=2e-4, mu=0.5)
    dhat = params["dhat"]
    rng = np.random.default_rng(seed)
    lx, ly, lz = 0.20, 0.002, 0.15
    nx, nz = plate_cells
    pv, pt = box_surface(lx, ly, lz, nx, 1, nz)
    tilt = math.radians(2.0 * (1 if rng.uniform() < 0.5 else -1) + rng.uniform(-0.1, 0.1))
    c, s = math.cos(tilt), math.sin(tilt)
    Rz = np.array([[c, 0, -s], [0, 1, 0], [s, 0, c]])   # rotation in the x-z plane
    pv = pv @ Rz.T
    ext = np.abs(pv).max(0) + np.array([1e-3, 0.0, 1e-3])
    ext[1] = ly / 2                                     # cage faces coincide with plate faces
    pn, ptet, pgrid = grid_cage(-ext, ext, plate_cage)
    b = _Builder()
    b.add_embedded(pv, pt, pn, ptet, pgrid)
    r = 3e-3
    na, nu = tine_segs
    height = 0.15
    for row in (-1, 1):
        for k in range(n_tines):
            tv, tt = open_cylinder(r, height, na, nu)
            # rotate so that a generator faces the plate exactly
            yc = row * (ly / 2 + 0.5 * dhat + r)
            ang = -np.pi / 2 if row > 0 else np.pi / 2
            ca, sa = math.cos(ang), math.sin(ang)
            tv = tv @ np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1]]).T
            xc = -0.1125 + 0.025 * k
            tv = tv + np.array([xc, yc, -0.10])
            b.add_kinematic(tv, tt)
    sc = b.scene("plate_in_rack", params)
    q_rest = sc.q_rest.copy()
    z_off = 0.055

    def q_at(t: float) -> np.ndarray:
        q = q_rest.copy()
        q[:, 2] += z_off - lower_per_iter * t
        return q

    def dq_at(t: int) -> np.ndarray:
        # next lowering step plus a sideways push of 0.75 dhat toward one tine row (the
        # gap is 0.5 dhat, so contact comes at two thirds of the step)
        d = q_at(float(t) + 1.0) - q_at(float(t))
        d[:, 1] += 0.75 * dhat
        return d

    sc.n_iterates = n_iters
    sc.iterate = lambda t: q_at(float(t))
    sc.lag_of = lambda t: (t // 5) * 5
    sc.dq = dq_at
    return sc


def _grid_dims(n_nodes: float, ext) -> Tuple[int, int, int]:
    """Cube counts (c_x, c_y, c_z) of a cage grid over a box with extents `ext` whose node
    count prod(c_i + 1) is closest to n_nodes (in ratio), for near-cubic cells."""
    ext = np.asarray(ext, float)
    target = max(float(n_nodes), 8.0)
    best, best_err = (1, 1, 1), np.inf
    for h in np.geomspace(ext.max(), ext.min() / 64.0, 2000):
        dims = tuple(int(max(1, round(e / h))) for e in ext)
        err = abs(np.log(np.prod(np.array(dims) + 1.0) / target))
        if err < best_err:
            best, best_err = dims, err
    return best


def batched_grasp(n_scenes: int = 256, seed: int = 0, min_tris: int = 2000, max_tris: int = 50000,
                  spacing: float = 0.2) -> Scene:
    """`n_scenes` independent bubble-grasp scenes concatenated into one (disjoint vertex and
    cage-node ranges; `body` holds each vertex's scene id).  Scene s has a total surface size
    log-uniform in [min_tris, max_tris] (half body, a quarter per membrane), cages of about
    one node per 40 surface vertices, and its own closing phase (a multiple of 3 iterates, so
    every scene's friction lags on the same iterates); scenes sit on a grid `spacing` apart.
    iterate(t) / dq(t) concatenate each scene's iterate / direction at its own phase + t."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in range(n_scenes):
        T = float(np.exp(rng.uniform(np.log(min_tris), np.log(max_tris))))
        nb = max(4, int(round(np.sqrt(T / 2 / 20))))
        nm = max(3, int(round(np.sqrt(T / 4 / 20))))
        body_nodes = 10 * nb * nb / 40.0
        mem_nodes = 10 * nm * nm / 40.0
        bc = _grid_dims(body_nodes, (0.11, 0.11, 0.11))
        mc = _grid_dims(mem_nodes, (0.123, 0.033, 0.083))
        sc = bubble_grasp(seed=seed * 100003 + s, n_body=nb, n_mem=nm, body_cage=bc, mem_cage=mc)
        phase = 3 * int(rng.integers(0, sc.n_iterates // 3))
        parts.append((sc, phase))
    g = int(np.ceil(n_scenes ** (1.0 / 3.0)))
    tris, cage_idx, w, xk, body, nodes, tets = [], [], [], [], [], [], []
    v_off = 0
    n_off = 0
    offsets = []
    for s, (sc, phase) in enumerate(parts):
        o = spacing * np.array([s % g, (s // g) % g, s // (g * g)], float)
        offsets.append((n_off, sc.Ns, o))
        tris.append(sc.tris + v_off)
        idx = sc.cage_idx.copy()
        idx[idx >= 0] += n_off
        cage_idx.append(idx)
        w.append(sc.w)
        xk.append(np.where(sc.kinematic[:, None], sc.x_kin + o, 0.0))
        body.append(np.full(sc.Nv, s, np.int32))
        nodes.append(sc.q_rest + o)
        tets.append(sc.cage_tets + n_off)
        v_off += sc.Nv
        n_off += sc.Ns
    tris = np.ascontiguousarray(np.concatenate(tris).astype(np.int32))
    out = Scene(name="batched_grasp", tris=tris, edges=edges_of(tris),
                cage_idx=np.ascontiguousarray(np.concatenate(cage_idx)), w=np.ascontiguousarray(np.concatenate(w)),
                x_kin=np.ascontiguousarray(np.concatenate(xk)), Ns=n_off, cage_tets=np.concatenate(tets),
                q_rest=np.ascontiguousarray(np.concatenate(nodes)), body=np.concatenate(body),
                params=dict(parts[0][0].params))
    n_it = parts[0][0].n_iterates

    def cat(fn, t):
        q = np.zeros((n_off, 3))
        for (sc, phase), (no, ns, o) in zip(parts, offsets):
            q[no:no + ns] = fn(sc, (phase + t) % n_it) + o
        return q

    def cat_dq(t):
        q = np.zeros((n_off, 3))
        for (sc, phase), (no, ns, o) in zip(parts, offsets):
            q[no:no + ns] = sc.dq((phase + t) % n_it)
        return q

    out.n_iterates = n_it
    out.iterate = lambda t: cat(lambda sc, tt: sc.iterate(tt), t)
    out.lag_of = parts[0][0].lag_of
    out.dq = cat_dq
    out.parts = parts
    out.n_scenes = n_scenes
    out.node_ranges = [(no, ns) for no, ns, _ in offsets]
    vr, fr, er = [], [], []
    v0 = f0 = 0
    for sc, _ in parts:
        vr.append((v0, sc.Nv)); fr.append((f0, sc.F))
        v0 += sc.Nv; f0 += sc.F
    # edges_of sorts rows lexicographically and the vertex ranges are increasing, so each
    # scene's edges form one contiguous run, in the scene's own order
    e0 = 0
    for sc, _ in parts:
        er.append((e0, sc.E)); e0 += sc.E
    out.vertex_ranges, out.tri_ranges, out.edge_ranges = vr, fr, er

    def part_scene(s: int) -> Scene:
        """Scene s alone, in the batch's coordinates (translated by its grid offset), so
        that its positions are bitwise those of its vertices in the batch."""
        sc, phase = parts[s]
        no, ns, o = offsets[s]
        one = Scene(name=f"batched_grasp[{s}]", tris=sc.tris.copy(), edges=sc.edges.copy(),
                    cage_idx=sc.cage_idx.copy(), w=sc.w.copy(),
                    x_kin=np.ascontiguousarray(np.where(sc.kinematic[:, None], sc.x_kin + o, 0.0)),
                    Ns=sc.Ns, cage_tets=sc.cage_tets.copy(), q_rest=sc.q_rest + o,
                    body=sc.body.copy(), params=dict(sc.params))
        one.n_iterates = n_it
        one.iterate = lambda t: sc.iterate((phase + t) % n_it) + o
        one.lag_of = sc.lag_of
        one.dq = lambda t: sc.dq((phase + t) % n_it)
        return one

    out.part_scene = part_scene
    return out


def parallel_sheets(seed: int = 0, cells: int = 12, angle_deg: float = 0.5, gap_frac: float = 0.5) -> Scene:
    """Two triangulated 2 x 2 cm sheets, a kinematic one at z = 0 and an embedded one
    (in a one-cube-thick cage) gap_frac dhat above it, turned by angle_deg in its plane, so
    that many edge-edge pairs within dhat are nearly parallel (the case the EE mollifier
    treats).  Cage nodes get N(0, 1 um) jitter; a second iterate slides the upper sheet by
    a seeded 0.2 dhat in-plane step.  dhat = 1e-3, mu = 0.5."""
    params = dict(DEFAULT_PARAMS)
    dhat = params["dhat"]
    rng = np.random.default_rng(seed)
    h = 0.01
    lv, lt = grid_plane(cells, cells, -h, h, -h, h)
    uv, ut = grid_plane(cells, cells, -0.9 * h, 0.9 * h, -0.9 * h, 0.9 * h)
    a = np.deg2rad(angle_deg)
    R = np.array([[np.cos(a), -np.sin(a), 0.0], [np.sin(a), np.cos(a), 0.0], [0.0, 0.0, 1.0]])
    uv = uv @ R.T
    uv[:, 2] = gap_frac * dhat
    nodes, tets, grid = grid_cage(uv.min(0) - np.array([1e-3, 1e-3, 5e-4]), uv.max(0) + np.array([1e-3, 1e-3, 5e-4]),
                                  (6, 6, 1))
    b = _Builder()
    b.add_embedded(uv, ut[:, [0, 2, 1]], nodes, tets, grid)
    b.add_kinematic(lv, lt)
    sc = b.scene("parallel_sheets", params)
    q0 = sc.q_rest + rng.normal(0.0, 1e-6, size=sc.q_rest.shape)
    step = np.zeros_like(q0)
    step[:, :2] = rng.normal(size=2) / np.sqrt(2.0) * 0.2 * dhat
    its = [q0, q0 + step]
    sc.n_iterates = 2
    sc.iterate = lambda t: its[t].copy()
    sc.lag_of = lambda t: 0
    sc.dq = lambda t: np.tile(np.array([0.0, 0.0, -2.0 * dhat]), (sc.Ns, 1))
    return sc


def pad_lift(seed: int = 0, small: bool = False, n_steps: int = 20, theta: float = 1e-4) -> Scene:
    """The sphere-on-pad scene as a dynamic trajectory: the cage is linear corotational
    (E = 5e4 Pa, nu = 0.45, rho = 1e3 kg/m^3, the soft body of Sec. IV-A) under gravity,
    its top layer of nodes held fixed; the kinematic pad moves up by `theta` per time step
    (h = 1e-2 s) for `n_steps` steps; checkpoints every 5 steps.  Inputs only: the driver
    and the adjoint read these attributes.
      q0            starting (and rest) cage positions, zero initial velocity
      fixed_nodes   bool [Ns], the top cage layer
      material      dict(E, nu, rho)
      gravity       [3] m/s^2
      pad_dir       unit direction of the pad motion; the pad at step n sits at
                    x_kin + n * theta * pad_dir
    small=True: level-2 icosphere, 3^3 cage cubes, 12 x 12 pad (for CPU tests)."""
    if small:
        sc = sphere_on_pad(seed, level=2, pad_cells=12, cage_cubes=3)
    else:
        sc = sphere_on_pad(seed)
    sc.name = "pad_lift" + ("_small" if small else "")
    sc.q0 = sc.iterate(0)
    ztop = sc.q_rest[:, 2].max()
    sc.fixed_nodes = np.abs(sc.q_rest[:, 2] - ztop) < 1e-12
    sc.material = dict(E=5e4, nu=0.45, rho=1e3)
    sc.gravity = np.array([0.0, 0.0, -9.81])
    sc.pad_dir = np.array([0.0, 0.0, 1.0])
    sc.theta = float(theta)
    sc.n_steps = int(n_steps)
    sc.checkpoint_every = 5
    return sc


def make_config(k: int, seed: int = 0, small: bool = False) -> Scene:
    """k = 1: sphere on pad; 2: bubble grasp; 3: plate in rack; 4: 256 batched bubble grasps;
    5: the sphere on a rising pad, a 20-step dynamic trajectory (the adjoint's workload).
    small=True gives reduced versions (configs 2 and 3 that the brute-force oracle enumerates
    in seconds; 16 small scenes for config 4; a coarse sphere for config 5)."""
    if k == 1:
        return sphere_on_pad(seed)
    if k == 5:
        return pad_lift(seed, small=small)
    if k == 2:
        if small:
            return bubble_grasp(seed, n_body=16, n_mem=10, body_cage=(5, 5, 5), mem_cage=(8, 3, 6))
        return bubble_grasp(seed)
    if k == 4:
        if small:
            return batched_grasp(n_scenes=16, seed=seed, min_tris=2000, max_tris=8000)
        return batched_grasp(n_scenes=256, seed=seed)
    if k == 3:
        if small:
            return plate_in_rack(seed, plate_cells=(40, 30), n_tines=4, tine_segs=(16, 20),
                                 plate_cage=(7, 1, 7), n_iters=20)
        return plate_in_rack(seed)
    raise ValueError(k)
