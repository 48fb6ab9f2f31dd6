"""Seeded synthetic particle clouds shaped like the paper's workloads.

This module only *produces inputs*: lattice positions with jitter, particle
types, normals, smoothing lengths, masses and smooth test fields.  It holds none
of the method's arithmetic (no neighbour search, PCA, stencils or remap), so
both the CUDA path and the CPU oracle may consume what it generates.

Shapes (all lengths in metres, h = 3.5 dx everywhere, jitter +-0.1 dx):

* ``cube_on_sheet``  -- a 3D cube resting on a one-layer film sheet, the
  cube's footprint removed from the sheet (Sec. 7.1 / 7.3 style geometry).
* ``jet_on_plate``   -- a vertical 3D cylinder standing on a plate, feeding a
  radial one-layer film disc (the cleaning-jet shape of Sec. 7.3).
* ``shallow_layer``  -- a shallow 3D layer in a box or cylinder, thin compared
  with h (the steady shallow-cylinder experiment of Sec. 7.1).

Particle types follow Sec. 2.3: 3D particles touching the plate are WALL, 3D
particles on exposed faces are FREE_SURFACE, the rest INTERIOR; film (2D)
particles are all WALL (Sec. 4.2).  Wall and film particles are jittered in
plane only, so they lie exactly on the plate.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2405_13165

MODEL_3D = 0
MODEL_2D = 1
TYPE_INTERIOR = 0
TYPE_FREE_SURFACE = 1
TYPE_WALL = 2

USER_TO_2D = 1  # bit set by a user-defined criterion requesting 3D -> 2D
USER_TO_3D = 2  # bit set by a user-defined criterion requesting 2D -> 3D

RHO_WATER = 1000.0   # Sec. 7.1
ETA_WATER = 1.0e-3   # Sec. 7.1


@dataclasses.dataclass
class Cloud:
    """Structure-of-arrays particle state (caller order)."""
    pos_h: np.ndarray    # float32 [N,4]  x, y, z, h
    model: np.ndarray    # uint8  [N]     MODEL_3D / MODEL_2D
    ptype: np.ndarray    # uint8  [N]     TYPE_*
    normal: np.ndarray   # float32 [N,4]  inward unit wall normal (0 if none)
    vp: np.ndarray       # float32 [N,4]  u, v, w, p  (velocity + pressure)
    rho: np.ndarray      # float32 [N]
    eta: np.ndarray      # float32 [N]
    mass: np.ndarray     # float32 [N]
    diam: np.ndarray     # float32 [N]    droplet diameter, V = pi d^3 / 6
    hfilm: np.ndarray    # float32 [N]    film height (2D particles)
    h3d: np.ndarray      # float32 [N]    user-prescribed 3D resolution
    user: np.ndarray     # uint8  [N]     USER_* bits
    last: np.ndarray     # uint8  [N]     1 if transitioned in previous step
    dx: float = 0.0
    name: str = ""
    # the modes of the sinusoid fields: (field, kappa_x, kappa_y, kappa_z, phi) each
    field_modes: tuple = ()

    @property
    def n(self) -> int:
        return int(self.pos_h.shape[0])

    @property
    def vol(self) -> np.ndarray:
        """Particle volume V = m / rho (= pi d^3 / 6 for droplets)."""
        return (self.mass.astype(np.float64) / self.rho.astype(np.float64)).astype(np.float32)

    @property
    def fields(self) -> np.ndarray:
        return self.vp

    def take(self, idx: np.ndarray) -> "Cloud":
        kw = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            kw[f.name] = np.ascontiguousarray(v[idx]) if isinstance(v, np.ndarray) else v
        return Cloud(**kw)

    def arrays(self) -> dict:
        return {f.name: getattr(self, f.name) for f in dataclasses.fields(self)
                if isinstance(getattr(self, f.name), np.ndarray)}


def concat(clouds: list[Cloud], name: str = "") -> Cloud:
    kw = {}
    for f in dataclasses.fields(Cloud):
        vals = [getattr(c, f.name) for c in clouds]
        if isinstance(vals[0], np.ndarray):
            kw[f.name] = np.ascontiguousarray(np.concatenate(vals, axis=0))
        elif f.name == "field_modes":
            kw[f.name] = vals[0] if all(v == vals[0] for v in vals) else ()
        else:
            kw[f.name] = vals[0]
    kw["name"] = name
    return Cloud(**kw)


def sinusoid_fields(xyz: np.ndarray, rng: np.random.Generator, modes: int = 4,
                    kmin: float = 1.0, kmax: float = 8.0, modes_out: list | None = None
                    ) -> np.ndarray:
    """u, v, w, p = sum of `modes` sinusoids sin(kappa . x + phi).

    kappa has a direction uniform on the sphere and |kappa| ~ U[kmin, kmax]
    (rad/m); phi ~ U[0, 2 pi).  Returns float32 [N,4]; with `modes_out`, also
    appends (field, kappa_x, kappa_y, kappa_z, phi) of every mode to it.
    """
    out = np.zeros((xyz.shape[0], 4), dtype=np.float64)
    for f in range(4):
        for _ in range(modes):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            k = d * rng.uniform(kmin, kmax)
            phi = rng.uniform(0.0, 2.0 * math.pi)
            out[:, f] += np.sin(xyz @ k + phi)
            if modes_out is not None:
                modes_out.append((f, float(k[0]), float(k[1]), float(k[2]), float(phi)))
    return out.astype(np.float32)


def _finish(xyz: np.ndarray, model: np.ndarray, ptype: np.ndarray, normal: np.ndarray,
            film_h: float, dx: float, rng: np.random.Generator, name: str) -> Cloud:
    n = xyz.shape[0]
    h = 3.5 * dx
    pos_h = np.empty((n, 4), dtype=np.float32)
    pos_h[:, :3] = xyz.astype(np.float32)
    pos_h[:, 3] = np.float32(h)
    rho = np.full(n, RHO_WATER, dtype=np.float32)
    eta = np.full(n, ETA_WATER, dtype=np.float32)
    vol = np.where(model == MODEL_3D, dx ** 3, dx * dx * film_h)
    mass = (RHO_WATER * vol).astype(np.float32)
    diam = np.cbrt(6.0 * vol / math.pi).astype(np.float32)
    hfilm = np.where(model == MODEL_2D, film_h, 0.0).astype(np.float32)
    modes: list = []
    vp = sinusoid_fields(pos_h[:, :3].astype(np.float64), rng, modes_out=modes)
    return Cloud(pos_h=pos_h, model=model.astype(np.uint8), ptype=ptype.astype(np.uint8),
                 normal=normal.astype(np.float32), vp=vp, rho=rho, eta=eta, mass=mass,
                 diam=diam, hfilm=hfilm, h3d=np.full(n, h, dtype=np.float32),
                 user=np.zeros(n, np.uint8), last=np.zeros(n, np.uint8), dx=dx, name=name,
                 field_modes=tuple(modes))


def _jitter(xyz: np.ndarray, planar: np.ndarray, dx: float, rng: np.random.Generator) -> np.ndarray:
    j = rng.uniform(-0.1 * dx, 0.1 * dx, size=xyz.shape)
    j[planar, 2] = 0.0
    return xyz + j


def cube_on_sheet(dx: float = 0.02, cube: float = 0.3, sheet: float = 1.0,
                  film_h_factor: float = 0.3, seed: int = SEED_BASE + 1) -> Cloud:
    """3D cube (edge `cube`) resting on a one-layer film sheet (edge `sheet`).

    The cube is centred on the sheet; its bottom layer (z = 0) is 3D WALL with
    normal +z, its side and top layers FREE_SURFACE, the rest INTERIOR.  Film
    particles share the cube's lattice in x/y; those under the cube's footprint
    are removed.
    """
    rng = np.random.default_rng(seed)
    m = int(round(cube / dx))
    s = int(round(sheet / dx))
    off = (s - m) // 2
    # cube lattice indices (i, j, k); film lattice indices (i, j)
    ii, jj, kk = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    cx = (off + ii + 0.5) * dx
    cy = (off + jj + 0.5) * dx
    cz = kk * dx
    ctype = np.full(ii.shape, TYPE_INTERIOR, np.uint8)
    face = (ii == 0) | (ii == m - 1) | (jj == 0) | (jj == m - 1) | (kk == m - 1)
    ctype[face] = TYPE_FREE_SURFACE
    ctype[kk == 0] = TYPE_WALL
    fi, fj = np.meshgrid(np.arange(s), np.arange(s), indexing="ij")
    fi, fj = fi.ravel(), fj.ravel()
    keep = ~((fi >= off) & (fi < off + m) & (fj >= off) & (fj < off + m))
    fi, fj = fi[keep], fj[keep]
    fx = (fi + 0.5) * dx
    fy = (fj + 0.5) * dx
    xyz = np.concatenate([np.stack([cx, cy, cz], 1), np.stack([fx, fy, np.zeros_like(fx)], 1)])
    model = np.concatenate([np.full(cx.shape, MODEL_3D), np.full(fx.shape, MODEL_2D)]).astype(np.uint8)
    ptype = np.concatenate([ctype, np.full(fx.shape, TYPE_WALL, np.uint8)])
    planar = ptype == TYPE_WALL
    normal = np.zeros((xyz.shape[0], 4), np.float32)
    normal[planar, 2] = 1.0
    xyz = _jitter(xyz, planar, dx, rng)
    return _finish(xyz, model, ptype, normal, film_h_factor * dx, dx, rng,
                   f"cube_on_sheet(dx={dx:g})")


def _jet_lattice(dx: float, r_cyl: float, height: float, r_film: float, plate: float):
    c = 0.5 * plate
    nr = int(math.floor(r_cyl / dx))
    ii, jj = np.meshgrid(np.arange(-nr, nr + 1), np.arange(-nr, nr + 1), indexing="ij")
    rr = np.hypot(ii * dx, jj * dx)
    inside = rr <= r_cyl
    ring = inside & (rr > r_cyl - dx)
    nk = int(math.floor(height / dx)) + 1
    nf = int(math.floor(r_film / dx))
    fi, fj = np.meshgrid(np.arange(-nf, nf + 1), np.arange(-nf, nf + 1), indexing="ij")
    fr = np.hypot(fi * dx, fj * dx)
    film = (fr <= r_film) & (fr > r_cyl)
    return c, ii[inside], jj[inside], ring[inside], nk, fi[film], fj[film]


def jet_on_plate_count(dx: float, r_cyl: float = 0.05, height: float = 0.5,
                       r_film: float = 1.0, plate: float = 2.0) -> int:
    _, ci, _, _, nk, fi, _ = _jet_lattice(dx, r_cyl, height, r_film, plate)
    return int(ci.size * nk + fi.size)


def jet_on_plate(dx: float | None = 0.004, n_target: int | None = None, r_cyl: float = 0.05,
                 height: float = 0.5, r_film: float = 1.0, plate: float = 2.0,
                 film_h_factor: float = 0.3, seed: int = SEED_BASE + 2) -> Cloud:
    """Vertical 3D cylinder (radius r_cyl, height) on a plate, radial film disc.

    If `n_target` is given, dx is bisected (shape ratios kept) until the
    particle count is within 1 % of it.
    """
    if n_target is not None:
        lo, hi = 1e-4, 0.05
        for _ in range(60):
            mid = math.sqrt(lo * hi)
            cnt = jet_on_plate_count(mid, r_cyl, height, r_film, plate)
            if abs(cnt - n_target) <= 0.01 * n_target:
                break
            if cnt > n_target:
                lo = mid
            else:
                hi = mid
        dx = mid
    rng = np.random.default_rng(seed)
    c, ci, cj, ring, nk, fi, fj = _jet_lattice(dx, r_cyl, height, r_film, plate)
    kk = np.repeat(np.arange(nk)[None, :], ci.size, 0).ravel()
    cii = np.repeat(ci, nk)
    cjj = np.repeat(cj, nk)
    rng_ring = np.repeat(ring, nk)
    cx = c + cii * dx
    cy = c + cjj * dx
    cz = kk * dx
    ctype = np.full(cx.shape, TYPE_INTERIOR, np.uint8)
    ctype[rng_ring | (kk == nk - 1)] = TYPE_FREE_SURFACE
    ctype[kk == 0] = TYPE_WALL
    fx = c + fi * dx
    fy = c + fj * dx
    xyz = np.concatenate([np.stack([cx, cy, cz], 1), np.stack([fx, fy, np.zeros_like(fx)], 1)])
    model = np.concatenate([np.full(cx.shape, MODEL_3D), np.full(fx.shape, MODEL_2D)]).astype(np.uint8)
    ptype = np.concatenate([ctype, np.full(fx.shape, TYPE_WALL, np.uint8)])
    planar = ptype == TYPE_WALL
    normal = np.zeros((xyz.shape[0], 4), np.float32)
    normal[planar, 2] = 1.0
    xyz = _jitter(xyz, planar, dx, rng)
    return _finish(xyz, model, ptype, normal, film_h_factor * dx, dx, rng,
                   f"jet_on_plate(dx={dx:.6g})")


def shallow_layer(dx: float, depth_layers: int, extent: float, cylinder: bool = True,
                  h_factor: float = 3.5, seed: int = SEED_BASE + 7, jitter: bool = True) -> Cloud:
    """Shallow 3D layer standing on a floor, in a cylinder (or square box).

    Floor layer: WALL, normal +z.  Side-wall ring (cylinder) or side faces
    (box): WALL with a horizontal inward normal.  Top layer: FREE_SURFACE.
    Everything else INTERIOR.  Used for the steady shallow-cylinder checks of
    Sec. 7.1 (floor particles transition, side-wall particles do not).
    """
    rng = np.random.default_rng(seed)
    n = int(round(extent / dx))
    ii, jj = np.meshgrid(np.arange(-n, n + 1), np.arange(-n, n + 1), indexing="ij")
    x = ii.ravel() * dx
    y = jj.ravel() * dx
    if cylinder:
        r = np.hypot(x, y)
        keep = r <= extent + 1e-9
        x, y, r = x[keep], y[keep], r[keep]
        side = r > extent - dx + 1e-9
        nrm_xy = -np.stack([x, y], 1) / np.maximum(r, 1e-30)[:, None]
    else:
        side = (np.abs(x) > extent - dx / 2) | (np.abs(y) > extent - dx / 2)
        nrm_xy = np.zeros((x.size, 2))
        nrm_xy[np.abs(x) > extent - dx / 2, 0] = -np.sign(x[np.abs(x) > extent - dx / 2])
        nrm_xy[np.abs(y) > extent - dx / 2, 1] = -np.sign(y[np.abs(y) > extent - dx / 2])
        nn = np.linalg.norm(nrm_xy, axis=1)
        nrm_xy[nn > 0] /= nn[nn > 0, None]
    xs, ys, zs, ts, ns = [], [], [], [], []
    for k in range(depth_layers):
        t = np.full(x.shape, TYPE_INTERIOR, np.uint8)
        nr = np.zeros((x.size, 3))
        if k == depth_layers - 1:
            t[:] = TYPE_FREE_SURFACE
        t[side] = TYPE_WALL
        nr[side, :2] = nrm_xy[side]
        if k == 0:
            t[:] = TYPE_WALL
            nr[~side] = (0.0, 0.0, 1.0)
            nr[side, :2] = nrm_xy[side]
        xs.append(x); ys.append(y); zs.append(np.full(x.shape, k * dx)); ts.append(t); ns.append(nr)
    xyz = np.stack([np.concatenate(xs), np.concatenate(ys), np.concatenate(zs)], 1)
    ptype = np.concatenate(ts)
    nrm = np.concatenate(ns)
    floor = (np.abs(xyz[:, 2]) < 1e-12)
    if jitter:
        j = rng.uniform(-0.1 * dx, 0.1 * dx, size=xyz.shape)
        j[floor, 2] = 0.0
        xyz = xyz + j
    normal = np.zeros((xyz.shape[0], 4), np.float32)
    normal[:, :3] = nrm
    model = np.full(xyz.shape[0], MODEL_3D, np.uint8)
    c = _finish(xyz, model, ptype, normal, 0.0, dx, rng, f"shallow_layer(dx={dx:g})")
    c.pos_h[:, 3] = np.float32(h_factor * dx)
    c.h3d[:] = np.float32(h_factor * dx)
    return c


def flat_film(dx: float, extent: float, film_h: float, seed: int = SEED_BASE + 8,
              jitter: bool = True, h_factor: float = 3.5) -> Cloud:
    """Single layer of 2D film particles on z = 0 over [0, extent]^2."""
    rng = np.random.default_rng(seed)
    n = int(round(extent / dx))
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    xyz = np.stack([(ii.ravel() + 0.5) * dx, (jj.ravel() + 0.5) * dx, np.zeros(ii.size)], 1)
    if jitter:
        j = rng.uniform(-0.1 * dx, 0.1 * dx, size=xyz.shape)
        j[:, 2] = 0.0
        xyz = xyz + j
    model = np.full(xyz.shape[0], MODEL_2D, np.uint8)
    ptype = np.full(xyz.shape[0], TYPE_WALL, np.uint8)
    normal = np.zeros((xyz.shape[0], 4), np.float32)
    normal[:, 2] = 1.0
    c = _finish(xyz, model, ptype, normal, film_h, dx, rng, f"flat_film(dx={dx:g})")
    c.pos_h[:, 3] = np.float32(h_factor * dx)
    c.h3d[:] = np.float32(h_factor * dx)
    return c


def rotation(axis, angle: float) -> np.ndarray:
    """3x3 rotation matrix about the unit direction of `axis` by `angle` (rad)."""
    k = np.asarray(axis, np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def rotated(cloud: Cloud, axis=(1.0, 0.4, 0.0), angle: float = 0.5) -> Cloud:
    """The cloud turned rigidly about `axis` through the origin (positions and
    normals; positions rounded to float32 again, so a tilted film is planar
    only up to that rounding)."""
    R = rotation(axis, angle)
    c = cloud.take(np.arange(cloud.n))
    c.pos_h[:, :3] = (cloud.pos_h[:, :3].astype(np.float64) @ R.T).astype(np.float32)
    c.normal[:, :3] = (cloud.normal[:, :3].astype(np.float64) @ R.T).astype(np.float32)
    c.name = f"rotated({cloud.name})"
    return c


def curved_film(dx: float, r_disc: float, radius: float, film_h: float | None = None,
                seed: int = SEED_BASE + 9, h_factor: float = 3.5) -> Cloud:
    """One layer of 2D film particles on a spherical cap: the points of a square
    lattice (u, v) at spacing dx within the disc u^2 + v^2 <= r_disc^2 (r_disc <
    radius), jittered +-0.1 dx in u and v, lifted to z = R - sqrt(R^2 - u^2 - v^2)
    (on the sphere of radius R centred at (0, 0, R)); inward normal towards the
    centre."""
    assert 0.0 < r_disc < radius
    rng = np.random.default_rng(seed)
    n = int(math.floor(r_disc / dx))
    ii, jj = np.meshgrid(np.arange(-n, n + 1), np.arange(-n, n + 1), indexing="ij")
    u0, v0 = ii.ravel() * dx, jj.ravel() * dx
    keep = u0 * u0 + v0 * v0 <= (r_disc - 0.1 * dx) ** 2
    u0, v0 = u0[keep], v0[keep]
    u = u0 + rng.uniform(-0.1 * dx, 0.1 * dx, u0.size)
    v = v0 + rng.uniform(-0.1 * dx, 0.1 * dx, v0.size)
    z = radius - np.sqrt(radius * radius - u * u - v * v)
    xyz = np.stack([u, v, z], 1)
    ctr = np.array([0.0, 0.0, radius])
    nrm = (ctr[None, :] - xyz) / np.linalg.norm(ctr[None, :] - xyz, axis=1)[:, None]
    model = np.full(xyz.shape[0], MODEL_2D, np.uint8)
    ptype = np.full(xyz.shape[0], TYPE_WALL, np.uint8)
    normal = np.zeros((xyz.shape[0], 4), np.float32)
    normal[:, :3] = nrm
    c = _finish(xyz, model, ptype, normal, 0.3 * dx if film_h is None else film_h, dx, rng,
                f"curved_film(dx={dx:g}, R={radius:g})")
    c.pos_h[:, 3] = np.float32(h_factor * dx)
    c.h3d[:] = np.float32(h_factor * dx)
    return c


def random_cloud(n: int, seed: int, box: float = 1.0, h_lo: float = 0.08, h_hi: float = 0.12,
                 frac2d: float = 0.3) -> Cloud:
    """Unstructured cloud with variable h and random models/types (edge cases)."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0, box, size=(n, 3))
    model = (rng.uniform(size=n) < frac2d).astype(np.uint8)
    xyz[model == MODEL_2D, 2] = 0.0
    ptype = rng.integers(0, 3, size=n).astype(np.uint8)
    ptype[model == MODEL_2D] = TYPE_WALL
    normal = np.zeros((n, 4), np.float32)
    normal[:, 2] = 1.0
    c = _finish(xyz, model, ptype, normal, 0.01, box / max(n, 1) ** (1 / 3), rng, f"random({n})")
    c.pos_h[:, 3] = rng.uniform(h_lo, h_hi, size=n).astype(np.float32)
    c.h3d[:] = c.pos_h[:, 3]
    return c


def config_small(seed: int = SEED_BASE + 1) -> Cloud:
    """Cube 0.3^3 at dx = 0.02 on a 1 x 1 film sheet (about 5.65k particles)."""
    return cube_on_sheet(0.02, seed=seed)


def config_jet_1m(seed: int = SEED_BASE + 2) -> Cloud:
    """Jet-on-plate cloud with dx bisected to 1M particles (within 1 %)."""
    return jet_on_plate(None, n_target=1_000_000, seed=seed)


def config_diff_2m(seed: int = SEED_BASE + 4) -> Cloud:
    """Cube-on-sheet shape with dx bisected to 2M particles (within 1 %)."""
    lo, hi = 1e-3, 0.02
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        m = int(round(0.3 / mid))
        s = int(round(1.0 / mid))
        cnt = m ** 3 + s * s - m * m
        if abs(cnt - 2_000_000) <= 20_000:
            break
        if cnt > 2_000_000:
            lo = mid
        else:
            hi = mid
    return cube_on_sheet(mid, seed=seed)


def batched_sizes(nclouds: int = 256, n_lo: int = 2_000, n_hi: int = 200_000,
                  film_lo: float = 0.1, film_hi: float = 0.9,
                  seed: int = SEED_BASE + 3) -> tuple[np.ndarray, np.ndarray]:
    """The draws behind `batched_clouds`: target sizes N_b and film fractions f_b."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=nclouds))
    films = rng.uniform(film_lo, film_hi, size=nclouds)
    return sizes, films


def batched_clouds(nclouds: int = 256, n_lo: int = 2_000, n_hi: int = 200_000,
                   film_lo: float = 0.1, film_hi: float = 0.9, dx: float = 0.02,
                   seed: int = SEED_BASE + 3, select=None) -> list[Cloud]:
    """Independent cube-on-sheet clouds of uneven size and model mix.

    Cloud b draws N_b log-uniform in [n_lo, n_hi] and a film fraction f_b
    uniform in [film_lo, film_hi] (from `seed`), then sizes the shape at the
    spacing dx: cube edge m = round(((1 - f_b) N_b)^(1/3)) cells, sheet edge
    s = round(sqrt(f_b N_b + m^2)) cells.  Its lattice, jitter and fields use
    seed 1000 * 3 + b above the base seed.  Every cloud sits at the same place,
    so clouds overlap in space and only the batching keeps them apart.
    select: the indices b to build (default all), each cloud as in the full batch.
    """
    sizes, films = batched_sizes(nclouds, n_lo, n_hi, film_lo, film_hi, seed)
    out = []
    for b in (range(nclouds) if select is None else select):
        m = max(2, int(round(((1.0 - films[b]) * sizes[b]) ** (1.0 / 3.0))))
        s = max(m + 2, int(round(math.sqrt(films[b] * sizes[b] + m * m))))
        out.append(cube_on_sheet(dx, cube=m * dx, sheet=s * dx, seed=SEED_BASE + 3 * 1000 + b))
    return out


def config_batched(nclouds: int = 256, select=None, **kw) -> tuple[Cloud, np.ndarray]:
    """The batched workload: `batched_clouds` each put in its own cell order and
    stored back to back; returns (cloud, int64 offsets [clouds + 1]).  select:
    only those clouds (in the given order), e.g. one rank's share."""
    parts = [cell_sorted(c) for c in batched_clouds(nclouds, select=select, **kw)]
    off = np.zeros(len(parts) + 1, np.int64)
    off[1:] = np.cumsum([c.n for c in parts])
    return concat(parts, f"batched({len(parts)} clouds)"), off


# ------------------------------------------------------- model interface strip
QUAD_FIELDS = np.array([       # u, v, w, p = c0 + c1 x + c2 y + c3 x^2 + c4 x y + c5 y^2
    [1.0, 2.0, -1.0, 0.5, 1.0, -0.3],
    [-0.5, 0.3, 0.8, -1.2, 0.4, 0.9],
    [0.2, -1.0, 0.5, 0.7, -0.6, 0.25],
    [3.0, 0.1, 0.2, 0.05, 0.8, -0.4]])


def interface_strip(dx: float = 0.02, layers: int = 3, extent=(1.0, 0.5), x_split: float = 0.5,
                    quadratic: bool = False, columns: bool = False,
                    seed: int = SEED_BASE + 6) -> Cloud:
    """Film (2D) for x < x_split and a 3D layer of `layers` particles for
    x >= x_split, side by side on the plate (the two-model arrangement of the
    advection tests of Sec. 7.2).  The film height is (layers - 1) dx, so a
    film particle lifted to 3D (Alg. 4, psi~ = dx) matches the layer.  3D
    particles in layer 0 are WALL, the top layer and the columns at the strip's
    edges FREE_SURFACE.  quadratic: fields are the depth-constant quadratics of
    QUAD_FIELDS instead of sinusoids; columns: every 3D column shares one
    in-plane jitter (vertical columns), otherwise the usual jitter."""
    rng = np.random.default_rng(seed)
    ni, nj = int(round(extent[0] / dx)), int(round(extent[1] / dx))
    I, J = np.meshgrid(np.arange(ni), np.arange(nj), indexing="ij")
    I, J = I.ravel(), J.ravel()
    x = (I + 0.5) * dx
    film = x < x_split
    fi, fj = I[film], J[film]
    ci, cj = I[~film], J[~film]
    k = np.repeat(np.arange(layers)[None, :], ci.size, 0).ravel()
    ci, cj = np.repeat(ci, layers), np.repeat(cj, layers)
    col_id = np.repeat(np.arange(ci.size // layers), layers)
    edge = (cj == 0) | (cj == nj - 1) | (ci == ci.min()) | (ci == ni - 1)
    ctype = np.where(k == 0, TYPE_WALL,
                     np.where((k == layers - 1) | edge, TYPE_FREE_SURFACE, TYPE_INTERIOR))
    xyz = np.concatenate([np.stack([(ci + 0.5) * dx, (cj + 0.5) * dx, k * dx], 1),
                          np.stack([(fi + 0.5) * dx, (fj + 0.5) * dx, np.zeros(fi.size)], 1)])
    model = np.concatenate([np.full(ci.size, MODEL_3D), np.full(fi.size, MODEL_2D)]).astype(np.uint8)
    ptype = np.concatenate([ctype, np.full(fi.size, TYPE_WALL)]).astype(np.uint8)
    planar = ptype == TYPE_WALL
    normal = np.zeros((xyz.shape[0], 4), np.float32)
    normal[planar, 2] = 1.0
    if columns:
        # in-plane jitter shared by each 3D column (columns stay vertical)
        cj_xy = rng.uniform(-0.1 * dx, 0.1 * dx, size=(col_id.max() + 1, 2))
        fj_xy = rng.uniform(-0.1 * dx, 0.1 * dx, size=(fi.size, 2))
        xyz[:, :2] += np.concatenate([cj_xy[col_id], fj_xy])
    else:
        xyz = _jitter(xyz, planar, dx, rng)
    c = _finish(xyz, model, ptype, normal, (layers - 1) * dx, dx, rng,
                f"interface_strip(dx={dx:g}, layers={layers})")
    if quadratic:
        X = c.pos_h[:, 0].astype(np.float64)
        Y = c.pos_h[:, 1].astype(np.float64)
        mono = np.stack([np.ones_like(X), X, Y, X * X, X * Y, Y * Y], 1)
        c.vp = (mono @ QUAD_FIELDS.T).astype(np.float32)
    return c


# --------------------------------------------------- advection-diffusion plate
ADV_DISC = (0.5, 0.5, 0.2)        # (x0, y0, radius) of the initial hot disc (Sec. 7.2)


def advection_plate(h: float, extent=(4.0, 3.0), seed: int = SEED_BASE + 7) -> Cloud:
    """The advection-diffusion plate of Sec. 7.2, all film (2D) at the start:
    film particles on [0, 4] x [0, 3] at spacing dx = h / 3.5 with film height
    2 dx (a film particle lifted to 3D by Alg. 4 becomes a column of three),
    temperature T in the first field slot: 1 inside the disc ADV_DISC, else 0
    (constant through the depth); the other field slots are 0."""
    dx = h / 3.5
    rng = np.random.default_rng(seed)
    ni, nj = int(round(extent[0] / dx)), int(round(extent[1] / dx))
    I, J = np.meshgrid(np.arange(ni), np.arange(nj), indexing="ij")
    xyz = np.stack([(I.ravel() + 0.5) * dx, (J.ravel() + 0.5) * dx, np.zeros(I.size)], 1)
    n = xyz.shape[0]
    model = np.full(n, MODEL_2D, np.uint8)
    ptype = np.full(n, TYPE_WALL, np.uint8)
    normal = np.zeros((n, 4), np.float32)
    normal[:, 2] = 1.0
    xyz = _jitter(xyz, np.ones(n, bool), dx, rng)
    c = _finish(xyz, model, ptype, normal, 2.0 * dx, dx, rng, f"advection_plate(h={h:g})")
    x0, y0, r = ADV_DISC
    P = c.pos_h.astype(np.float64)
    inside = (P[:, 0] - x0) ** 2 + (P[:, 1] - y0) ** 2 <= r * r
    c.vp = np.zeros((n, 4), np.float32)
    c.vp[:, 0] = inside.astype(np.float32)
    return c


# ---------------------------------------------------------------- tray loop
TRAY_SHEET = (2.0, 1.0)          # film sheet extent (m)
TRAY_JET_FOOT = (0.45, 0.5)      # where the jet axis meets the plate
TRAY_JET_TILT = math.radians(30.0)
TRAY_JET_R, TRAY_JET_LEN = 0.02, 0.3
TRAY_BLOBS = 256


def _tray_heights(dx: float, rng: np.random.Generator) -> np.ndarray:
    """Puddle depth in layers per film site: the largest of TRAY_BLOBS Gaussian
    bumps (amplitude U[2, 8] dx, sigma U[10, 40] dx, cut at 3 sigma), rounded
    to whole layers; blobs keep clear of the jet foot."""
    ni, nj = int(round(TRAY_SHEET[0] / dx)), int(round(TRAY_SHEET[1] / dx))
    H = np.zeros((ni, nj), np.float32)
    placed = 0
    while placed < TRAY_BLOBS:
        cx = rng.uniform(0.1, TRAY_SHEET[0] - 0.1)
        cy = rng.uniform(0.1, TRAY_SHEET[1] - 0.1)
        sig = rng.uniform(10.0, 40.0) * dx
        amp = rng.uniform(2.0, 8.0)
        if math.hypot(cx - TRAY_JET_FOOT[0], cy - TRAY_JET_FOOT[1]) < 3.0 * sig + 0.2:
            continue
        placed += 1
        i0, i1 = max(0, int((cx - 3 * sig) / dx)), min(ni, int((cx + 3 * sig) / dx) + 1)
        j0, j1 = max(0, int((cy - 3 * sig) / dx)), min(nj, int((cy + 3 * sig) / dx) + 1)
        xs = (np.arange(i0, i1) + 0.5) * dx - cx
        ys = (np.arange(j0, j1) + 0.5) * dx - cy
        r2 = xs[:, None] ** 2 + ys[None, :] ** 2
        bump = amp * np.exp(-r2 / (2.0 * sig * sig))
        bump[r2 > 9.0 * sig * sig] = 0.0
        np.maximum(H[i0:i1, j0:j1], bump.astype(np.float32), out=H[i0:i1, j0:j1])
    return np.floor(H + 0.5).astype(np.int32)


def _tray_jet(dx: float):
    """Lattice sites (i, j, k) of the inclined jet column (axis tilted from the
    vertical towards +x, ending on the plate) and their free-surface flags."""
    a = np.array([math.sin(TRAY_JET_TILT), 0.0, math.cos(TRAY_JET_TILT)])
    fx, fy = TRAY_JET_FOOT
    r, L = TRAY_JET_R, TRAY_JET_LEN
    i0 = int((fx - r) / dx) - 1
    i1 = int((fx + L * a[0] + r) / dx) + 2
    j0, j1 = int((fy - r) / dx) - 1, int((fy + r) / dx) + 2
    nk = int((L * a[2] + r) / dx) + 2
    X = (np.arange(i0, i1) + 0.5) * dx - fx
    Y = (np.arange(j0, j1) + 0.5) * dx - fy
    I, J = np.meshgrid(X, Y, indexing="ij")
    occ = np.zeros((I.shape[0], I.shape[1], nk), bool)
    for k in range(nk):                     # one layer at a time (bounded memory)
        Z = k * dx
        s = I * a[0] + J * a[1] + Z * a[2]
        rad2 = (I - s * a[0]) ** 2 + (J - s * a[1]) ** 2 + (Z - s * a[2]) ** 2
        occ[:, :, k] = (rad2 <= r * r) & (s <= L)
    pad = np.zeros((occ.shape[0] + 2, occ.shape[1] + 2, occ.shape[2] + 2), bool)
    pad[1:-1, 1:-1, 1:-1] = occ
    pad[1:-1, 1:-1, 0] = True                     # the plate below layer 0
    exposed = np.zeros_like(occ)
    for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        exposed |= ~pad[1 + d[0]:pad.shape[0] - 1 + d[0], 1 + d[1]:pad.shape[1] - 1 + d[1],
                        1 + d[2]:pad.shape[2] - 1 + d[2]]
    oi, oj, ok = np.nonzero(occ)
    return oi + i0, oj + j0, ok, exposed[oi, oj, ok]


def tray_count(dx: float, seed: int = SEED_BASE + 5) -> int:
    rng = np.random.default_rng(seed)
    L = _tray_heights(dx, rng)
    ji, jj, jk, _ = _tray_jet(dx)
    foot = np.zeros_like(L, bool)
    ok = (jk == 0) & (ji >= 0) & (ji < L.shape[0]) & (jj >= 0) & (jj < L.shape[1])
    foot[ji[ok], jj[ok]] = True
    return int(L.sum() + ji.size + ((L == 0) & ~foot).sum())


def tray_cloud(dx: float, film_h_factor: float = 0.3, seed: int = SEED_BASE + 5) -> Cloud:
    """Tray-cleaning shape: a 2 x 1 m film sheet with pooled 3D puddles (columns
    under Gaussian bumps up to 8 layers) and an inclined 3D jet column
    (r = 0.02 m, 0.3 m long, 30 degrees from the vertical) standing on it.
    3D particles in layer 0 are WALL, those with an empty lattice neighbour (or
    the top of a column) FREE_SURFACE, the rest INTERIOR; film sites under 3D
    matter are removed."""
    rng = np.random.default_rng(seed)
    L = _tray_heights(dx, rng)
    ni, nj = L.shape
    # puddle columns
    ci, cj = np.nonzero(L > 0)
    Lc = L[ci, cj]
    rep = np.repeat(np.arange(ci.size), Lc)
    pk = np.arange(rep.size) - np.repeat(np.cumsum(Lc) - Lc, Lc)
    pi, pj = ci[rep], cj[rep]
    Lp = np.pad(L, 1)
    side = np.minimum.reduce([Lp[pi, pj + 1], Lp[pi + 2, pj + 1], Lp[pi + 1, pj], Lp[pi + 1, pj + 2]])
    ptype = np.where(pk == 0, TYPE_WALL,
                     np.where((pk == L[pi, pj] - 1) | (side <= pk), TYPE_FREE_SURFACE,
                              TYPE_INTERIOR)).astype(np.uint8)
    # jet column
    ji, jj, jk, jexp = _tray_jet(dx)
    jtype = np.where(jk == 0, TYPE_WALL,
                     np.where(jexp, TYPE_FREE_SURFACE, TYPE_INTERIOR)).astype(np.uint8)
    foot = np.zeros_like(L, bool)
    ok = (jk == 0) & (ji >= 0) & (ji < ni) & (jj >= 0) & (jj < nj)
    foot[ji[ok], jj[ok]] = True
    fi, fj = np.nonzero((L == 0) & ~foot)
    xyz = np.concatenate([
        np.stack([(pi + 0.5) * dx, (pj + 0.5) * dx, pk * dx], 1),
        np.stack([(ji + 0.5) * dx, (jj + 0.5) * dx, jk * dx], 1),
        np.stack([(fi + 0.5) * dx, (fj + 0.5) * dx, np.zeros(fi.size)], 1)])
    model = np.concatenate([np.full(pi.size, MODEL_3D), np.full(ji.size, MODEL_3D),
                            np.full(fi.size, MODEL_2D)]).astype(np.uint8)
    ptype = np.concatenate([ptype, jtype, np.full(fi.size, TYPE_WALL, np.uint8)])
    planar = ptype == TYPE_WALL
    normal = np.zeros((xyz.shape[0], 4), np.float32)
    normal[planar, 2] = 1.0
    xyz = _jitter(xyz, planar, dx, rng)
    return _finish(xyz, model, ptype, normal, film_h_factor * dx, dx, rng,
                   f"tray(dx={dx:.6g})")


def config_tray(n_target: int = 16_000_000, seed: int = SEED_BASE + 5) -> Cloud:
    """Tray shape with dx bisected to n_target particles (within 1 %), in cell order."""
    lo, hi = 2e-4, 0.01
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        cnt = tray_count(mid, seed)
        if abs(cnt - n_target) <= 0.01 * n_target:
            break
        if cnt > n_target:
            lo = mid
        else:
            hi = mid
    return cell_sorted(tray_cloud(mid, seed=seed))


def tray_velocity(dx: float, seed: int = SEED_BASE + 5 * 1000) -> dict:
    """Smooth random displacement field of the tray loop (float32 parameters):
    d(x) = sum_m a_m e_m b(u_m),  u_m = frac((kappa_m . x + phi_m) / (2 pi)),
    b(u) = 16 u^2 (1 - u)^2 - 16/30 (a C2-periodic, zero-mean bump), four
    modes with e_m and kappa_m uniform on the sphere, |kappa_m| ~ U[2, 10]
    rad/m, amplitudes scaled so that |d| <= 0.2 dx per step.  Built from +, *
    and floor only, so float32 evaluations agree bit for bit on any IEEE
    device when the operations are taken in the stated order."""
    rng = np.random.default_rng(seed)
    e = rng.normal(size=(4, 3))
    e /= np.linalg.norm(e, axis=1, keepdims=True)
    k = rng.normal(size=(4, 3))
    k /= np.linalg.norm(k, axis=1, keepdims=True)
    k *= rng.uniform(2.0, 10.0, size=(4, 1))
    phi = rng.uniform(0.0, 2.0 * math.pi, size=4)
    a = rng.uniform(0.5, 1.0, size=4)
    a *= 0.2 * dx / (a.sum() * (16.0 / 30.0))     # |b| <= 16/30
    f32 = np.float32
    return {"e": e.astype(f32), "kappa": k.astype(f32), "phi": phi.astype(f32),
            "amp": a.astype(f32), "inv_2pi": f32(1.0 / (2.0 * math.pi)),
            "mean": f32(16.0 / 30.0), "zmin": f32(0.5 * dx)}


def tray_sphere(step: int) -> tuple[np.ndarray, float, float]:
    """User criterion of the tray loop (a sphere on the plate sweeping along x,
    like the distance criterion of Sec. 7.4): (centre, radius, trailing shell).
    Film particles inside the sphere are asked to become 3D; 3D particles in
    the shell it has just left are asked to become 2D."""
    c = np.array([0.15 + 0.09 * step, 0.5, 0.0])
    return c, 0.2, 0.09


def cell_order(pos_h: np.ndarray, cell_factor: float = 1.0 + 1e-6) -> np.ndarray:
    """Cell order of a cloud: cells of edge max(h) * cell_factor from the
    bounding-box minimum, keys (cz * ny + cy) * nx + cx, stable in index;
    returns the permutation (sorted position -> index).

    A Lagrangian code keeps its particles in this order between steps; it is
    the order the neighbour search's own cell sort produces, so a cloud in it
    takes the search's sorted path.  Input layout only (no method arithmetic).
    """
    P = pos_h.astype(np.float64)
    lo = P[:, :3].min(0)
    hi = P[:, :3].max(0)
    c = float(P[:, 3].max()) * cell_factor
    inv_c = 1.0 / c
    dim = np.floor((hi - lo) / c) + 1.0
    cc = np.floor((P[:, :3] - lo) * inv_c)
    cc = np.clip(cc, 0, dim - 1).astype(np.int64)
    key = (cc[:, 2] * int(dim[1]) + cc[:, 1]) * int(dim[0]) + cc[:, 0]
    return np.argsort(key, kind="stable")


def cell_sorted(cloud: Cloud, cell_factor: float = 1.0 + 1e-6) -> Cloud:
    """The cloud permuted into cell order (see cell_order)."""
    return cloud.take(cell_order(cloud.pos_h, cell_factor))
