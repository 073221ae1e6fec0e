"""The synthetic workloads HRPP is measured and checked on.

The paper's scenes (Teapot, Killeroo, Buddha, Sportscar; Table 1) are not
available, so seeded procedural scenes of a similar range of triangle counts
stand in for them.  Every array is made by `scenes` (scenegen.c) from the seeds
given here.

  small_scene   icosphere (3x subdivided, 1,280 triangles, radius 1, centre
                (0,1,0)) on a 16x16-quad ground grid over [-4,4]^2 (512
                triangles); binary BVH, <= 4 triangles per leaf; 256x256
                pinhole primary rays from (0,2.5,6) toward (0,0.75,0), 45 deg
                vertical field of view; one shadow ray per hit toward a point
                light at (2,4,2); predictor 2^12 entries, direct-mapped.
  terrain_scene value-noise terrain of 708x708 quads over [-50,50]^2 (1,002,528
                triangles; 4 octaves, amplitude 8, base frequency 1/16) with 64
                icospheres (5x subdivided, 20,480 triangles each, radius
                log-uniform in [0.1, 2]) resting on it: 2,313,248 triangles;
                4-wide BVH; 1920x1080 primary closest-hit rays from (0,25,-70)
                toward the origin, 60 deg field of view; 4 cosine-weighted
                ambient-occlusion any-hit rays per hit, tmax 0.5.
Both take size parameters so tests can run the same recipe at reduced size.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

from . import (ao_rays, build_bvh, icosphere, pinhole_rays, place_spheres, quad_grid, shadow_rays,
               soup, sphere_rays, terrain)


@dataclass
class Scene:
    name: str
    tris: np.ndarray       # float32 [n, 9]
    nodes: np.ndarray      # NODE_DTYPE [m]
    prim_index: np.ndarray  # uint32 [n]
    root: int
    width: int
    camera: dict

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    def primary_rays(self, frame: int = 0, seed: int | None = None) -> np.ndarray:
        c = self.camera
        return pinhole_rays(c["eye"], c["target"], c["vfov"], c["width"], c["height"],
                            seed=c["seed"] if seed is None else seed, frame=frame)


def small_scene(width: int = 2, subdiv: int = 3, grid: int = 16, res: int = 256) -> Scene:
    sphere = icosphere(subdiv, (0.0, 1.0, 0.0), 1.0)
    ground = quad_grid(grid, grid, -4.0, 4.0, -4.0, 4.0, 0.0)
    tris = np.ascontiguousarray(np.concatenate([sphere, ground]), np.float32)
    nodes, prim, root = build_bvh(tris, width=width)
    cam = dict(eye=(0.0, 2.5, 6.0), target=(0.0, 0.75, 0.0), vfov=45.0, width=res, height=res, seed=0)
    return Scene("small", tris, nodes, prim, root, width, cam)


SMALL_LIGHT = (2.0, 4.0, 2.0)
# A low point light beside the terrain (an evening sun): the shadows of its
# hills and spheres cover 86 % of the frame's hit points, the simple-lighting
# regime in which the paper finds hit-any locality (Sec. 6.1).
TERRAIN_SUN = (-80.0, 8.0, 0.0)


def terrain_scene(quads: int = 708, n_spheres: int = 64, subdiv: int = 5, width: int = 4, seed: int = 2,
                  res=(1920, 1080), extent: float = 50.0) -> Scene:
    ground = terrain(quads, quads, -extent, extent, -extent, extent, seed)
    parts = [ground]
    if n_spheres:
        sp = place_spheres(n_spheres, seed, 0.1, 2.0, -extent, extent, -extent, extent, seed)
        for cx, cy, cz, r in sp:
            parts.append(icosphere(subdiv, (float(cx), float(cy), float(cz)), float(r)))
    tris = np.ascontiguousarray(np.concatenate(parts), np.float32)
    nodes, prim, root = build_bvh(tris, width=width)
    cam = dict(eye=(0.0, 25.0, -70.0), target=(0.0, 0.0, 0.0), vfov=60.0, width=res[0], height=res[1], seed=seed)
    return Scene("terrain", tris, nodes, prim, root, width, cam)


def secondary_shadow(scene: Scene, rays: np.ndarray, hit_t, hit_prim, light=SMALL_LIGHT):
    """Shadow rays from the hits of `rays` (hit_t, hit_prim: closest-hit result)."""
    return shadow_rays(rays, hit_t, hit_prim, scene.tris, light)


def secondary_ao(scene: Scene, rays: np.ndarray, hit_t, hit_prim, frame: int = 0, per_hit: int = 4,
                 tmax: float = 0.5):
    """Cosine-weighted ambient-occlusion rays from the hits of `rays`."""
    return ao_rays(rays, hit_t, hit_prim, scene.tris, per_hit=per_hit, tmax=tmax,
                   seed=scene.camera["seed"], frame=frame)


# ------------------------------------------------------------ batched --

def _camera_for(tris: np.ndarray):
    v = tris.reshape(-1, 3)
    lo, hi = v.min(0).astype(np.float64), v.max(0).astype(np.float64)
    c = 0.5 * (lo + hi)
    ext = float(np.max(hi - lo))
    eye = c + ext * np.array([0.35, 0.9, -1.7])
    return tuple(eye), tuple(c), lo, hi


def batched_item(kind: str, n_tris: int, n_rays: int, seed: int, width: int = 4) -> tuple:
    """One scene of the batched workload and its rays.

    kind: 'terrain' (value-noise quad grid over [-1,1]^2, amplitude 0.16),
    'spheres' (icospheres of 320 triangles, centres uniform in [0,1]^3), or
    'soup' (uniform triangle soup in the unit cube).  Rays: half from a
    pinhole camera outside the scene looking at its centre, half with origins
    uniform in the scene's box and directions uniform on the sphere."""
    rng = np.random.default_rng(seed)
    if kind == "terrain":
        q = max(2, int(round(np.sqrt(n_tris / 2))))
        tris = terrain(q, q, -1.0, 1.0, -1.0, 1.0, seed, amp=0.16, freq=1.0 / 0.32)
    elif kind == "spheres":
        m = max(1, n_tris // 320)
        r = 0.35 * m ** (-1.0 / 3.0)
        cs = rng.uniform(r, 1 - r, (m, 3))
        tris = np.concatenate([icosphere(2, tuple(c), r) for c in cs])
    else:
        tris = soup(n_tris, seed)
    tris = np.ascontiguousarray(tris, np.float32)
    nodes, prim, root = build_bvh(tris, width=width)
    eye, tgt, lo, hi = _camera_for(tris)
    n_cam = n_rays // 2
    w = max(1, int(np.ceil(np.sqrt(n_cam * 16 / 9))))
    h = max(1, int(np.ceil(n_cam / w)))
    s = Scene(f"{kind}{seed}", tris, nodes, prim, root, width,
              dict(eye=eye, target=tgt, vfov=60.0, width=w, height=h, seed=seed))
    return s, batched_rays(s, n_rays, 0)


def batched_rays(scene: Scene, n_rays: int, frame: int) -> np.ndarray:
    """The rays of a batched-workload scene for one frame: the camera half
    at pixel centres (frame 0) or jittered (frame > 0), the random half drawn
    from a stream of its own per frame."""
    cam = scene.camera
    _, _, lo, hi = _camera_for(scene.tris)
    n_cam = n_rays // 2
    c = pinhole_rays(cam["eye"], cam["target"], cam["vfov"], cam["width"], cam["height"], seed=cam["seed"],
                     frame=frame)[:n_cam]
    rseed = cam["seed"] if frame == 0 else cam["seed"] + 7919 * frame
    rnd = sphere_rays(n_rays - n_cam, rseed, float(lo.min()), float(hi.max()))
    return np.ascontiguousarray(np.concatenate([c, rnd]), np.float32)


def batched_workload(n_scenes: int = 64, tris_range=(10_000, 2_000_000), rays_range=(4_096, 2_000_000),
                     seed: int = 3, width: int = 4):
    """The uneven batched workload: n_scenes scenes with log-uniform triangle
    counts in tris_range (terrain, icosphere clusters and triangle soup in
    turn) and log-uniform ray batch sizes in rays_range.  Yields (scene, rays)."""
    rng = np.random.default_rng(seed)
    kinds = ("terrain", "spheres", "soup")
    specs = []
    for k in range(n_scenes):
        nt = int(np.exp(rng.uniform(np.log(tris_range[0]), np.log(tris_range[1]))))
        nr = int(np.exp(rng.uniform(np.log(rays_range[0]), np.log(rays_range[1]))))
        specs.append((kinds[k % 3], nt, nr, seed * 1000 + k, width))
    # the items are independent and their generators and BVH builds run in C
    # outside the interpreter lock: build them on host threads, yield in order
    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        yield from ex.map(lambda a: batched_item(*a), specs)


# ------------------------------------------------------- path tracing --

PATH_LIGHT = (30.0, 80.0, -40.0)


def pathtrace_scene(quads=(2048, 1024), n_spheres: int = 256, subdiv: int = 2, width: int = 4, seed: int = 5,
                    res=(1280, 720), dome_subdiv: int = 4, dome_radius: float = 160.0) -> Scene:
    """Incoherent path-tracing scene: a value-noise terrain of quads[0] x
    quads[1] quads over [-100,100] x [-50,50] (4 octaves, amplitude 8, base
    frequency 1/16) with n_spheres icospheres (subdiv x subdivided, radius
    log-uniform in [0.1, 2]) resting on it, closed by a dome (an icosphere of
    radius dome_radius about the origin) so that no path escapes and every
    path runs all its bounces.  At the defaults: 4,194,304 + 81,920 + 5,120
    = 4,281,344 triangles."""
    nx, nz = quads
    ground = terrain(nx, nz, -100.0, 100.0, -50.0, 50.0, seed)
    parts = [ground]
    if dome_subdiv >= 0:
        parts.append(icosphere(dome_subdiv, (0.0, 0.0, 0.0), dome_radius))
    if n_spheres:
        sp = place_spheres(n_spheres, seed, 0.1, 2.0, -100.0, 100.0, -50.0, 50.0, seed)
        for cx, cy, cz, r in sp:
            parts.append(icosphere(subdiv, (float(cx), float(cy), float(cz)), float(r)))
    tris = np.ascontiguousarray(np.concatenate(parts), np.float32)
    nodes, prim, root = build_bvh(tris, width=width)
    cam = dict(eye=(0.0, 30.0, -90.0), target=(0.0, 0.0, 0.0), vfov=60.0, width=res[0], height=res[1], seed=seed)
    return Scene("pathtrace", tris, nodes, prim, root, width, cam)


def path_primary(scene: Scene, spp: int = 4, frame: int = 0) -> np.ndarray:
    """spp jittered samples per pixel: spp pinhole images concatenated."""
    return np.ascontiguousarray(np.concatenate([scene.primary_rays(frame=1 + spp * frame + k) for k in range(spp)]))


def path_bounces(scene: Scene, primary: np.ndarray, trace_closest, bounces: int = 5, light=PATH_LIGHT,
                 frame: int = 0):
    """Rays of a diffuse path tracer, bounce by bounce.

    trace_closest(rays) -> (t float32[n], prim uint32[n]) is the caller's
    closest-hit tracer (the oracle in tests, the library in benchmarks).
    Bounce b traces its closest-hit rays; each hit spawns one shadow ray
    toward the point light (any-hit) and one cosine-weighted diffuse ray
    (the next bounce).  Returns [(closest_rays_b, shadow_rays_b)]."""
    out = []
    rays = primary
    for b in range(bounces):
        t, p = trace_closest(rays)
        shadow, _ = shadow_rays(rays, t, p, scene.tris, light)
        out.append((rays, shadow))
        if b + 1 < bounces:
            rays, _ = ao_rays(rays, t, p, scene.tris, per_hit=1, tmax=float("inf"),
                              seed=scene.camera["seed"] + 7919 * (b + 1), frame=frame)
            if len(rays) == 0:
                break
    return out
