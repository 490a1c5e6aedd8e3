"""Seeded scene generators.

Every array is produced by numpy's PCG64 from an explicit seed, so a scene is
reproducible bit for bit on any host. Per-view inputs are generated lazily from
a child seed of (scene seed, view index): any single view can be rebuilt
without generating the others, which keeps the 300-view, 1920x1080 workload
out of host memory.

Recipes (the attribute laws of the workloads this library is measured on):

* Gaussian attributes: log-scales ~ N(-3.5, 0.3) per axis, turned into linear
  scales with exp in float64 and rounded to float32; unit quaternions (w, x, y,
  z) drawn as normalised 4-d normals; opacity = sigmoid(N(0, 1)).
* Means: uniform in [-1, 1]^3 ("uniform" scenes) or spread evenly over
  random ellipsoid surfaces ("surface" scenes): centres U[-0.6, 0.6]^3,
  semi-axes U[0.15, 0.45]^3, a random rotation; a point is the centre plus the
  rotated, axis-scaled image of a normalised 3-d normal direction.
* Cameras: pinhole, horizontal field of view 60 degrees, square pixels, the
  principal point at the image centre, on an orbit of radius 3 around the
  origin at elevation 0.3 rad with azimuth 2*pi*i/V; the jittered orbit adds
  N(0, 0.05) rad to azimuth and elevation, scales the radius by
  1 + U(-0.05, 0.05) and aims at N(0, 0.05)^3. Axes follow the OpenCV
  convention (x right, y down, z forward); R maps world to camera.
* Segment ids: a Voronoi partition of the image with K seeds uniform in pixel
  space; a pixel (x, y) takes the seed nearest to its centre (x + 0.5,
  y + 0.5) by squared distance, ties to the lower seed id.
* Segment embeddings: P prototype directions (unit normals in R^D); each
  segment picks a prototype uniformly, adds N(0, sigma) per coordinate and is
  renormalised to unit length.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Iterator, List, Optional

import numpy as np


# ----------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Gaussians:
    means: np.ndarray      # (N, 3) float32, world space
    scales: np.ndarray     # (N, 3) float32, linear (already exponentiated)
    quats: np.ndarray      # (N, 4) float32, (w, x, y, z)
    opacities: np.ndarray  # (N,)   float32, activated, in (0, 1)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Gaussians":
        return Gaussians(self.means[idx], self.scales[idx], self.quats[idx], self.opacities[idx])


@dataclasses.dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    R: np.ndarray          # (3, 3) float32, world -> camera, row-major
    t: np.ndarray          # (3,)   float32
    near: float = 0.01
    far: float = 100.0


@dataclasses.dataclass
class View:
    camera: Camera
    seg: np.ndarray        # (H, W) int32, -1 = pixel in no segment
    table: np.ndarray      # (M, D) float32, one embedding per segment id

    @property
    def m(self) -> int:
        return int(self.table.shape[0])


class Scene:
    """A Gaussian set plus a lazily generated list of views."""

    def __init__(self, name: str, gaussians: Gaussians, n_views: int,
                 view_fn: Callable[[int], View], dim: int, meta: Optional[dict] = None):
        self.name = name
        self.gaussians = gaussians
        self.n_views = n_views
        self._view_fn = view_fn
        self.dim = dim
        self.meta = dict(meta or {})

    def view(self, i: int) -> View:
        if not 0 <= i < self.n_views:
            raise IndexError(i)
        return self._view_fn(i)

    def views(self, idx=None) -> Iterator[View]:
        for i in (range(self.n_views) if idx is None else idx):
            yield self.view(i)


# ----------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------

def _rng(*keys: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(keys))))


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _attributes(rng: np.random.Generator, n: int):
    log_scales = rng.normal(-3.5, 0.3, size=(n, 3))
    scales = np.exp(log_scales).astype(np.float32)
    quats = _unit_quats(rng, n).astype(np.float32)
    opac = (1.0 / (1.0 + np.exp(-rng.standard_normal(n)))).astype(np.float32)
    return scales, quats, opac


def random_gaussians(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> Gaussians:
    """Means uniform in [lo, hi]^3 with the standard attribute laws."""
    rng = _rng(seed, 11)
    means = rng.uniform(lo, hi, size=(n, 3)).astype(np.float32)
    scales, quats, opac = _attributes(rng, n)
    return Gaussians(means, scales, quats, opac)


def _random_rotation_f64(rng: np.random.Generator) -> np.ndarray:
    # Orients the synthetic ellipsoid surfaces (input construction only):
    # Q factor of a 3x3 normal matrix with the signs of R's diagonal folded in.
    a = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def ellipsoid_gaussians(seed: int, n: int, n_surfaces: int) -> Gaussians:
    """Means spread evenly over `n_surfaces` random ellipsoid surfaces."""
    rng = _rng(seed, 12)
    centres = rng.uniform(-0.6, 0.6, size=(n_surfaces, 3))
    axes = rng.uniform(0.15, 0.45, size=(n_surfaces, 3))
    rots = [_random_rotation_f64(rng) for _ in range(n_surfaces)]
    counts = np.full(n_surfaces, n // n_surfaces)
    counts[: n % n_surfaces] += 1
    means = np.empty((n, 3))
    o = 0
    for s in range(n_surfaces):
        c = int(counts[s])
        u = rng.standard_normal((c, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        means[o:o + c] = centres[s] + (u * axes[s]) @ rots[s].T
        o += c
    scales, quats, opac = _attributes(rng, n)
    return Gaussians(means.astype(np.float32), scales, quats, opac)


def look_at(eye, target, width: int, height: int, fov_x_deg: float = 60.0,
            near: float = 0.01, far: float = 100.0) -> Camera:
    """Pinhole camera at `eye` aimed at `target`, world up = +z."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ eye
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(fx=float(np.float32(fx)), fy=float(np.float32(fx)),
                  cx=width / 2.0, cy=height / 2.0, width=int(width), height=int(height),
                  R=R.astype(np.float32), t=t.astype(np.float32), near=near, far=far)


def orbit_camera(i: int, n_views: int, width: int, height: int, radius: float = 3.0,
                 elevation: float = 0.3, jitter_rng: Optional[np.random.Generator] = None,
                 fov_x_deg: float = 60.0) -> Camera:
    az = 2.0 * math.pi * i / n_views
    el = elevation
    target = np.zeros(3)
    if jitter_rng is not None:
        az += jitter_rng.normal(0.0, 0.05)
        el += jitter_rng.normal(0.0, 0.05)
        radius = radius * (1.0 + jitter_rng.uniform(-0.05, 0.05))
        target = jitter_rng.normal(0.0, 0.05, size=3)
    eye = target + radius * np.array([math.cos(el) * math.cos(az),
                                      math.cos(el) * math.sin(az),
                                      math.sin(el)])
    return look_at(eye, target, width, height, fov_x_deg)


def voronoi_segments(rng: np.random.Generator, width: int, height: int, k: int) -> np.ndarray:
    """(H, W) int32 map: nearest of k uniform seeds to each pixel centre.

    Exact nearest-seed search by 32x32 pixel blocks: a seed can be nearest to a
    pixel of a block only if its distance to the block's box of pixel centres
    does not exceed the smallest, over all seeds, distance to the box's far
    corner; the distances of the remaining candidates are the same float64
    expressions as a search over all seeds, and ties still go to the lower id.
    """
    seeds = np.stack([rng.uniform(0, width, k), rng.uniform(0, height, k)], axis=1)
    return voronoi_from_seeds(seeds, width, height)


def voronoi_from_seeds(seeds: np.ndarray, width: int, height: int) -> np.ndarray:
    """(H, W) int32 map of the nearest of the given (k, 2) seeds (x, y), ties to the lower id."""
    seeds = np.asarray(seeds, np.float64)
    sx, sy = seeds[:, 0], seeds[:, 1]
    out = np.empty((height, width), np.int32)
    xs_all = np.arange(width, dtype=np.float64) + 0.5
    ys_all = np.arange(height, dtype=np.float64) + 0.5
    blk = 32
    for y0 in range(0, height, blk):
        ys = ys_all[y0:min(height, y0 + blk)]
        near_y = np.maximum(np.maximum(ys[0] - sy, sy - ys[-1]), 0.0)
        far_y = np.maximum(np.abs(sy - ys[0]), np.abs(sy - ys[-1]))
        dy = ys[:, None] - sy[None, :]
        dyy = dy * dy                                   # (rows, k)
        for x0 in range(0, width, blk):
            xs = xs_all[x0:min(width, x0 + blk)]
            near_x = np.maximum(np.maximum(xs[0] - sx, sx - xs[-1]), 0.0)
            far_x = np.maximum(np.abs(sx - xs[0]), np.abs(sx - xs[-1]))
            bound = (far_x * far_x + far_y * far_y).min()
            cand = np.nonzero(near_x * near_x + near_y * near_y <= bound * (1.0 + 1e-9) + 1e-9)[0]
            dx = xs[:, None] - sx[None, cand]           # (cols, candidates)
            d2 = dx[None, :, :] * dx[None, :, :] + dyy[:, None, cand]
            out[y0:y0 + len(ys), x0:x0 + len(xs)] = cand[np.argmin(d2, axis=2)]   # ties -> lower id
    return out


def prototype_table(rng: np.random.Generator, protos: np.ndarray, m: int, sigma: float) -> np.ndarray:
    pick = rng.integers(0, protos.shape[0], size=m)
    e = protos[pick] + rng.normal(0.0, sigma, size=(m, protos.shape[1]))
    e /= np.linalg.norm(e, axis=1, keepdims=True)
    return e.astype(np.float32)


def _prototypes(seed: int, p: int, d: int) -> np.ndarray:
    rng = _rng(seed, 13)
    v = rng.standard_normal((p, d))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

def make_scene(name: str, seed: int, gaussians: Gaussians, n_views: int, width: int, height: int,
               n_segments: int, n_protos: int, dim: int = 512, jitter: bool = False,
               noise_sigma: float = 0.1, empty_fraction: float = 0.0,
               resolutions: Optional[List[tuple]] = None, proto_seed: Optional[int] = None) -> Scene:
    """Scene with orbit cameras, Voronoi segment maps and prototype tables.

    `empty_fraction` > 0 marks that fraction of the Voronoi cells as "no
    segment" (id -1), to exercise unmasked pixels. `resolutions`, when given,
    assigns view i the resolution resolutions[i % len(resolutions)]. `proto_seed`, when given,
    draws the prototype directions of the scene made with that seed (the embedding law of
    another workload).
    """
    proto_seed = seed if proto_seed is None else proto_seed
    protos = _prototypes(proto_seed, n_protos, dim)

    def view_fn(i: int) -> View:
        rng = _rng(seed, 1000 + i)
        w, h = (resolutions[i % len(resolutions)] if resolutions else (width, height))
        cam = orbit_camera(i, n_views, w, h, jitter_rng=rng if jitter else None)
        seg = voronoi_segments(rng, w, h, n_segments)
        if empty_fraction > 0:
            drop = rng.uniform(size=n_segments) < empty_fraction
            seg = np.where(drop[seg], -1, seg).astype(np.int32)
        table = prototype_table(rng, protos, n_segments, noise_sigma)
        return View(cam, seg, table)

    return Scene(name, gaussians, n_views, view_fn, dim,
                 meta=dict(seed=seed, width=width, height=height, n_segments=n_segments,
                           n_protos=n_protos, jitter=jitter, noise_sigma=noise_sigma, proto_seed=proto_seed))


def config_tiny(seed: int = 0) -> Scene:
    """5,000 Gaussians uniform in [-1,1]^3, 4 views 128x128, 16 segments, 8 prototypes."""
    g = random_gaussians(seed, 5000)
    return make_scene("tiny", seed, g, n_views=4, width=128, height=128, n_segments=16, n_protos=8)


def config_mid(seed: int = 1) -> Scene:
    """300,000 Gaussians on 20 ellipsoids, 64 jittered views 960x540, 64 segments, 32 prototypes."""
    g = ellipsoid_gaussians(seed, 300_000, 20)
    return make_scene("mid", seed, g, n_views=64, width=960, height=540, n_segments=64,
                      n_protos=32, jitter=True)


def config_precision(seed: int = 2) -> Scene:
    """2,000,000 Gaussians on 60 ellipsoids, 300 jittered views 1920x1080, 128 segments, 64 prototypes."""
    g = ellipsoid_gaussians(seed, 2_000_000, 60)
    return make_scene("precision", seed, g, n_views=300, width=1920, height=1080, n_segments=128,
                      n_protos=64, jitter=True)


def config_learned(seed: int = 4, noise_sigma: float = 0.1) -> Scene:
    """The learned form's workload: 2,000,000 Gaussians on 60 ellipsoids, 300 jittered views
    1920x1080 with 128 segments, whose embeddings follow the mid-scale workload's law (its 32
    prototypes, made with seed 1, and N(0, noise_sigma) per coordinate): the law the latent
    form's autoencoder is trained on."""
    g = ellipsoid_gaussians(seed, 2_000_000, 60)
    return make_scene("learned", seed, g, n_views=300, width=1920, height=1080, n_segments=128,
                      n_protos=32, jitter=True, noise_sigma=noise_sigma, proto_seed=1)


def config_batched(seed: int = 3, n_scenes: int = 16) -> List[Scene]:
    """16 independent scenes: Gaussian counts log-uniform in [50k, 1.5M] on ellipsoid surfaces
    (one per 25k Gaussians), view counts uniform in [20, 200], resolutions drawn from
    {640x480, 960x540, 1920x1080}, 32..128 segments per view, D = 512, 32 prototypes."""
    rng = _rng(seed, 77)
    res = [(640, 480), (960, 540), (1920, 1080)]
    out = []
    for i in range(n_scenes):
        n = int(round(math.exp(rng.uniform(math.log(50_000), math.log(1_500_000)))))
        n_views = int(rng.integers(20, 201))
        w, h = res[int(rng.integers(0, 3))]
        m = int(rng.integers(32, 129))
        g = ellipsoid_gaussians(seed * 1000 + i, n, max(1, n // 25_000))
        out.append(make_scene(f"batched{i}", seed * 1000 + i, g, n_views=n_views, width=w, height=h,
                              n_segments=m, n_protos=32, jitter=True))
    return out


def small_scene(seed: int, n: int, n_views: int, width: int, height: int, n_segments: int,
                dim: int = 64, surfaces: int = 0, empty_fraction: float = 0.0,
                n_protos: int = 8, noise_sigma: float = 0.1) -> Scene:
    """Parity-test scene: sizes chosen so the oracle finishes in seconds."""
    g = ellipsoid_gaussians(seed, n, surfaces) if surfaces else random_gaussians(seed, n)
    return make_scene(f"small{seed}", seed, g, n_views=n_views, width=width, height=height,
                      n_segments=n_segments, n_protos=n_protos, dim=dim, jitter=True,
                      empty_fraction=empty_fraction, noise_sigma=noise_sigma)


def segment_samples(scene_seed: int, n: int, dim: int, n_protos: int, noise_sigma: float = 0.1,
                    sample_seed: int = 0) -> np.ndarray:
    """n segment embeddings drawn like the tables of the scene made with `scene_seed` (the
    same prototypes and noise law): training data for the latent form's autoencoder."""
    protos = _prototypes(scene_seed, n_protos, dim)
    return prototype_table(_rng(scene_seed, 50_000 + sample_seed), protos, n, noise_sigma)
