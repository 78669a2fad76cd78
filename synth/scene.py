"""Seeded procedural scenes shaped like the paper's workloads.

The paper measures on rasterised views of large indoor/outdoor scenes
(Section 3).  Those scenes are not available, so every workload here is a
room (12 triangles, normals facing inward) filled with randomly placed,
scaled and rotated icospheres and boxes.  All geometry is emitted as an
indexed float32 triangle mesh; that float32 array is the single canonical
input both the device path and the CPU checker read.

This module holds only scene construction (mesh generation, placement by
rejection of overlapping bounding spheres).  It computes no ray/triangle
intersection, no distance field and nothing of the query itself.
"""
from __future__ import annotations

import dataclasses
import functools
import math

import numpy as np

from . import rng

# Random streams (one per purpose so that changing one count never shifts another).
_S_PLACE = 1
_S_SIZE = 2
_S_ROT = 3
_S_BOXDIM = 4


@functools.lru_cache(maxsize=None)
def icosphere(subdiv: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere: icosahedron split `subdiv` times, vertices pushed to the sphere.

    Returns (V float64 (nv,3), F int32 (nf,3)); faces are counter-clockwise seen
    from outside (outward normals).  nf = 20 * 4**subdiv.
    """
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
         (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
         (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    faces = list(f)
    for _ in range(subdiv):
        mid: dict[tuple[int, int], int] = {}

        def midpoint(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                mid[key] = len(verts) - 1
            return mid[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts, dtype=np.float64)
    F = np.array(faces, dtype=np.int32)
    # orient outward: the signed volume of each face's tetrahedron with the centre is positive
    vol = np.einsum("ij,ij->i", V[F[:, 0]], np.cross(V[F[:, 1]], V[F[:, 2]]))
    flip = vol < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def box_mesh() -> tuple[np.ndarray, np.ndarray]:
    """Unit cube [-0.5, 0.5]^3 as 8 vertices and 12 outward-facing triangles."""
    V = np.array([[x, y, z] for z in (-0.5, 0.5) for y in (-0.5, 0.5) for x in (-0.5, 0.5)],
                 dtype=np.float64)
    # vertex index = x + 2y + 4z (bits)
    quads = [(0, 2, 3, 1),  # z = -0.5, normal -z
             (4, 5, 7, 6),  # z = +0.5, normal +z
             (0, 1, 5, 4),  # y = -0.5, normal -y
             (2, 6, 7, 3),  # y = +0.5, normal +y
             (0, 4, 6, 2),  # x = -0.5, normal -x
             (1, 3, 7, 5)]  # x = +0.5, normal +x
    F = []
    for a, b, c, d in quads:
        F += [(a, b, c), (a, c, d)]
    F = np.array(F, dtype=np.int32)
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    centroid = V[F].mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", n, centroid) > 0)
    return V, F


def room_mesh(W: float, H: float, D: float) -> tuple[np.ndarray, np.ndarray]:
    """Closed room [0,W]x[0,H]x[0,D]: the unit box scaled, with faces turned inward."""
    V, F = box_mesh()
    V = (V + 0.5) * np.array([W, H, D])
    return V, F[:, [0, 2, 1]].copy()


def quat_to_matrix(u1: float, u2: float, u3: float) -> np.ndarray:
    """Uniform random rotation from three uniforms (Shoemake, Graphics Gems III, 1992)."""
    a, b = math.sqrt(1 - u1), math.sqrt(u1)
    x, y = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    z, w = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


@dataclasses.dataclass
class SceneObject:
    kind: str                  # "sphere" | "box"
    center: np.ndarray         # (3,)
    radius: float              # sphere radius / box bounding-sphere radius
    rot: np.ndarray            # (3,3)
    extent: np.ndarray         # box edge lengths (3,); sphere: (2r, 2r, 2r)
    first_tri: int
    n_tris: int


@dataclasses.dataclass
class Camera:
    eye: np.ndarray
    forward: np.ndarray
    right: np.ndarray
    up: np.ndarray
    tan_half_fov: float
    width: int
    height: int


@dataclasses.dataclass
class SceneSpec:
    name: str
    room: tuple[float, float, float]
    n_spheres: int
    sphere_subdiv: int
    n_boxes: int
    grid_n: int
    scale_lo: float = 0.2        # log-uniform object scale (sphere diameter / box size)
    scale_hi: float = 2.0
    fixed_sphere_radius: float | None = None   # tiny config: one sphere of radius 0.6
    box_edge_uniform: tuple[float, float] | None = None  # tiny config: edges U(0.3, 1), axis-aligned
    rotate: bool = True
    resolution: tuple[int, int] = (1920, 1080)


@dataclasses.dataclass
class Scene:
    spec: SceneSpec
    seed: int
    verts: np.ndarray          # float32 (nv,3)
    tris: np.ndarray           # int32 (nt,3)
    objects: list[SceneObject]
    room: tuple[float, float, float]
    camera: Camera
    dropped: int               # objects that found no free position

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def lo(self) -> np.ndarray:
        return np.zeros(3, dtype=np.float32)

    @property
    def hi(self) -> np.ndarray:
        return np.array(self.room, dtype=np.float32)

    @property
    def diagonal(self) -> float:
        return float(np.linalg.norm(np.array(self.room, dtype=np.float64)))


# Workload shapes.  Triangle counts follow from the object counts:
# tiny 344; medium 25,732; frame 2,050,412; precision 8,201,612; fit 102,532.
SPECS = {
    "tiny": SceneSpec("tiny", (4.0, 3.0, 4.0), 1, 2, 1, 32, fixed_sphere_radius=0.6,
                      box_edge_uniform=(0.3, 1.0), rotate=False, resolution=(64, 64)),
    "medium": SceneSpec("medium", (8.0, 4.0, 8.0), 20, 3, 10, 64, scale_lo=0.3, scale_hi=1.5,
                        resolution=(160, 120)),
    "frame": SceneSpec("frame", (20.0, 6.0, 20.0), 400, 4, 200, 256),
    "precision": SceneSpec("precision", (40.0, 8.0, 40.0), 1600, 4, 800, 512),
    "fit": SceneSpec("fit", (10.0, 4.0, 10.0), 20, 4, 10, 128, resolution=(1024, 1024)),
}


def make_camera(room, width: int, height: int, vfov_deg: float = 60.0) -> Camera:
    W, H, D = room
    eye = np.array([0.5 * W, 0.55 * H, 0.06 * D])
    target = np.array([0.5 * W, 0.35 * H, 0.75 * D])
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return Camera(eye, fwd, right, up, math.tan(math.radians(vfov_deg) / 2), width, height)


def make_scene(name: str, seed: int = 2305) -> Scene:
    """Build the named workload scene from `seed` (deterministic on every platform)."""
    spec = SPECS[name]
    W, H, D = spec.room
    room = np.array(spec.room, dtype=np.float64)
    cam = make_camera(spec.room, *spec.resolution)

    # --- object sizes -----------------------------------------------------
    kinds = ["sphere"] * spec.n_spheres + ["box"] * spec.n_boxes
    n_obj = len(kinds)
    u_size = rng.uniform(seed, _S_SIZE, max(n_obj, 1))
    u_dim = rng.uniform(seed, _S_BOXDIM, 3 * max(n_obj, 1)).reshape(-1, 3)
    u_rot = rng.uniform(seed, _S_ROT, 3 * max(n_obj, 1)).reshape(-1, 3)
    objs = []
    for i, k in enumerate(kinds):
        if k == "sphere":
            if spec.fixed_sphere_radius is not None:
                r = spec.fixed_sphere_radius
            else:
                s = spec.scale_lo * (spec.scale_hi / spec.scale_lo) ** u_size[i]  # diameter
                r = 0.5 * s
            ext = np.array([2 * r] * 3)
            bound = r
        else:
            if spec.box_edge_uniform is not None:
                lo_e, hi_e = spec.box_edge_uniform
                ext = lo_e + (hi_e - lo_e) * u_dim[i]
            else:
                s = spec.scale_lo * (spec.scale_hi / spec.scale_lo) ** u_size[i]
                ext = s * (0.5 + 0.5 * u_dim[i])
            bound = 0.5 * float(np.linalg.norm(ext))
        R = quat_to_matrix(*u_rot[i]) if spec.rotate else np.eye(3)
        objs.append((i, k, bound, ext, R))
    # place larger objects first so that the packing by rejection succeeds
    order = sorted(range(n_obj), key=lambda j: -objs[j][2])

    # --- placement by rejection (bounding spheres must not overlap) -------
    placed_c = np.zeros((0, 3))
    placed_r = np.zeros((0,))
    gap = 0.02 * float(min(spec.room))
    keep_out = 0.3
    tries = 100
    u_pos = rng.uniform(seed, _S_PLACE, 3 * tries * max(n_obj, 1)).reshape(max(n_obj, 1), tries, 3)
    centers: dict[int, np.ndarray] = {}
    dropped = 0
    for j in order:
        _, k, r, ext, R = objs[j]
        span = room - 2 * (r + gap)
        if np.any(span <= 0):
            dropped += 1
            continue
        ok = None
        for t in range(tries):
            c = (r + gap) + u_pos[j, t] * span
            if np.linalg.norm(c - cam.eye) < r + keep_out:
                continue
            if placed_r.size and np.any(np.linalg.norm(placed_c - c, axis=1) < placed_r + r + gap):
                continue
            ok = c
            break
        if ok is None:
            dropped += 1
            continue
        centers[j] = ok
        placed_c = np.vstack([placed_c, ok])
        placed_r = np.append(placed_r, r)

    # --- emit the mesh ----------------------------------------------------
    Vs, Fs = [], []
    nv = 0
    rv, rf = room_mesh(W, H, D)
    Vs.append(rv)
    Fs.append(rf)
    nv += rv.shape[0]
    ntri = rf.shape[0]
    scene_objs = []
    for j in range(n_obj):
        if j not in centers:
            continue
        _, k, r, ext, R = objs[j]
        c = centers[j]
        if k == "sphere":
            V0, F0 = icosphere(spec.sphere_subdiv)
            V = (V0 * r) @ R.T + c
        else:
            V0, F0 = box_mesh()
            V = (V0 * ext) @ R.T + c
        Vs.append(V)
        Fs.append(F0 + nv)
        scene_objs.append(SceneObject(k, c, float(r), R, np.asarray(ext, dtype=np.float64), ntri, F0.shape[0]))
        nv += V.shape[0]
        ntri += F0.shape[0]
    verts = np.ascontiguousarray(np.concatenate(Vs).astype(np.float32))
    tris = np.ascontiguousarray(np.concatenate(Fs).astype(np.int32))
    return Scene(spec, seed, verts, tris, scene_objs, spec.room, cam, dropped)


def free_lights(scene: Scene, count: int = 4, below_ceiling: float = 0.4, clearance: float = 0.3) -> np.ndarray:
    """Point lights in free space under the ceiling: candidates on a 9 x 9 grid
    at below_ceiling under it, kept when `clearance` outside every object's
    bounding sphere; the one nearest to each quarter point of the room is taken.
    (count, 3) float64."""
    room = np.asarray(scene.room, dtype=np.float64)
    xs = np.linspace(0.1, 0.9, 9)
    cand = np.array([[x * room[0], room[1] - below_ceiling, z * room[2]] for x in xs for z in xs])
    ok = np.ones(len(cand), dtype=bool)
    for ob in scene.objects:
        ok &= np.linalg.norm(cand - np.asarray(ob.center), axis=1) > ob.radius + clearance
    cand = cand[ok]
    out = []
    for qx, qz in ((0.25, 0.25), (0.75, 0.25), (0.25, 0.75), (0.75, 0.75))[:count]:
        q = np.array([qx * room[0], room[1] - below_ceiling, qz * room[2]])
        out.append(cand[np.argmin(np.linalg.norm(cand - q, axis=1))])
    return np.array(out)
