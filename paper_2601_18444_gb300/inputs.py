"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *generates* real-space fields (cell positions, cell volumes,
nuclear densities N_j, magnetizations M_j, object offsets and centres,
rotation matrices).  It holds none of the SANS arithmetic: no Fourier sum, no
rotation of positions, no cross section.  Both the FP64 oracle (tests) and the
CUDA library are fed from here, so neither depends on the other.

Units: lengths in nm.  Every generator is deterministic in its ``seed``.

Workloads (paper sections they stand in for):
  * ``sphere_vortex``      -- uniform-N sphere with a vortex magnetization
                              (Sec. "Spherical form factor model" / linear vortex
                              and the runtime-experiment particle).
  * ``box_field``          -- micromagnetic-style box, smooth random M with pores
                              (stands in for MuMax3 output, Sec. on iron particles).
  * ``sphere_ensemble``    -- ragged ensemble of spheres with Neel-like canting
                              (the 800-particle interference example, scaled).
  * ``ellipsoid_uniform``  -- single-domain ellipsoid for rotational averaging.
  * ``random_rotations``   -- uniform random rotation matrices (Shoemake).
  * ``vortex_family``      -- the parameterised vortex particle of the surrogate.
"""
from __future__ import annotations

import numpy as np


class Field:
    """Real-space input of one SANS computation (host arrays, float64)."""

    def __init__(self, pos, vol, nuc, mag, offsets=None, centers=None, name=""):
        self.pos = np.ascontiguousarray(pos, dtype=np.float64)      # [n,3] nm
        self.vol = np.ascontiguousarray(vol, dtype=np.float64)      # [n]
        self.nuc = None if nuc is None else np.ascontiguousarray(nuc, dtype=np.float64)  # [n]
        self.mag = None if mag is None else np.ascontiguousarray(mag, dtype=np.float64)  # [n,3]
        self.offsets = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.int64)
        self.centers = None if centers is None else np.ascontiguousarray(centers, dtype=np.float64)
        self.name = name

    @property
    def n(self):
        return self.pos.shape[0]

    @property
    def n_objects(self):
        return 1 if self.offsets is None else len(self.offsets) - 1


def lattice_ball(radius, a, center_on_site=True):
    """Simple-cubic lattice sites (spacing a) inside a ball of given radius."""
    m = int(np.floor(radius / a)) + 1
    r = np.arange(-m, m + 1, dtype=np.float64) * a
    if not center_on_site:
        r = r + 0.5 * a
    x, y, z = np.meshgrid(r, r, r, indexing="ij")
    p = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    keep = (p ** 2).sum(1) <= radius * radius * (1.0 + 1e-12)
    return p[keep]


def _normalise(v):
    n = np.linalg.norm(v, axis=1, keepdims=True)
    n[n == 0] = 1.0
    return v / n


def sphere_vortex(radius=16.0, a=2.0, core=4.0, seed=0):
    """Sphere of radius R on a simple-cubic lattice, N_j = 1, |M_j| = 1.

    M is an in-plane curl of chirality c = +-1 plus a Gaussian core of width
    ``core`` along z with polarity p = +-1; c and p are drawn from ``seed``.
    """
    rng = np.random.default_rng(seed)
    c = 1.0 if rng.random() < 0.5 else -1.0
    p = 1.0 if rng.random() < 0.5 else -1.0
    pos = lattice_ball(radius, a)
    x, y = pos[:, 0], pos[:, 1]
    rho = np.hypot(x, y)
    safe = np.where(rho > 0, rho, 1.0)
    m = np.zeros_like(pos)
    m[:, 0] = np.where(rho > 0, -c * y / safe, 0.0)
    m[:, 1] = np.where(rho > 0, c * x / safe, 0.0)
    m[:, 2] = p * np.exp(-rho ** 2 / (2.0 * core * core))
    m = _normalise(m)
    n = pos.shape[0]
    return Field(pos, np.full(n, a ** 3), np.ones(n), m, name=f"sphere_vortex_R{radius}_a{a}")


def linear_vortex_sphere(radius=20.0, a=2.0, M0=1.0, M1=None, N0=1.0, normalised=False):
    """Sphere with M = M0 e_z + M1 (x e_y - y e_x) (linear vortex).

    With ``normalised`` the field is m = (-5y/R, 5x/R, 1)/norm, the particle of
    the runtime experiment (D = 40 nm, a = 2 nm gives 4169 cells).
    """
    if M1 is None:
        M1 = 5.0 * M0 / radius
    pos = lattice_ball(radius, a)
    x, y = pos[:, 0], pos[:, 1]
    m = np.stack([-M1 * y, M1 * x, np.full_like(x, M0)], axis=1)
    if normalised:
        m = _normalise(m)
    n = pos.shape[0]
    return Field(pos, np.full(n, a ** 3), np.full(n, N0), m, name="linear_vortex")


def box_field(nx=256, ny=256, nz=64, a=2.0, n_modes=64, kmax=0.2, n_pores=200,
              pore_r=(3.0, 8.0), seed=1, pores=True):
    """Micromagnetic-style box of nx*ny*nz cells (spacing a, centred).

    M = normalise(sum_m a_m cos(k_m . r + phi_m)) with |k_m| <= kmax uniform in
    the ball, a_m ~ N(0, I3), phi_m ~ U[0, 2pi).  N_j = 1.  Inside each of
    ``n_pores`` spherical pores (radius U[pore_r], centre uniform in the box)
    N_j = 0 and M_j = 0.
    """
    rng = np.random.default_rng(seed)
    ix = (np.arange(nx) - (nx - 1) / 2.0) * a
    iy = (np.arange(ny) - (ny - 1) / 2.0) * a
    iz = (np.arange(nz) - (nz - 1) / 2.0) * a
    X, Y, Z = np.meshgrid(ix, iy, iz, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    del X, Y, Z
    # wave vectors uniform in the ball of radius kmax
    d = rng.normal(size=(n_modes, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    kk = kmax * rng.random(n_modes) ** (1.0 / 3.0)
    kvec = d * kk[:, None]
    amp = rng.normal(size=(n_modes, 3))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    n = pos.shape[0]
    m = np.zeros((n, 3))
    step = 1 << 18
    for s in range(0, n, step):
        arg = pos[s:s + step] @ kvec.T + phi[None, :]
        m[s:s + step] = np.cos(arg) @ amp
    m = _normalise(m)
    nuc = np.ones(n)
    if pores and n_pores > 0:
        lo = pos.min(0)
        hi = pos.max(0)
        pc = lo + (hi - lo) * rng.random((n_pores, 3))
        pr = rng.uniform(pore_r[0], pore_r[1], size=n_pores)
        void = np.zeros(n, dtype=bool)
        # cells are on a lattice: visit only the bounding box of each pore
        shape = (nx, ny, nz)
        for c, r in zip(pc, pr):
            lo_i = np.maximum(np.floor((c - r - pos[0]) / a).astype(int), 0)
            hi_i = np.minimum(np.ceil((c + r - pos[0]) / a).astype(int) + 1, shape)
            gx = np.arange(lo_i[0], hi_i[0])
            gy = np.arange(lo_i[1], hi_i[1])
            gz = np.arange(lo_i[2], hi_i[2])
            if gx.size == 0 or gy.size == 0 or gz.size == 0:
                continue
            GX, GY, GZ = np.meshgrid(gx, gy, gz, indexing="ij")
            flat = (GX * ny + GY) * nz + GZ
            flat = flat.ravel()
            inside = ((pos[flat] - c) ** 2).sum(1) <= r * r
            void[flat[inside]] = True
        nuc[void] = 0.0
        m[void] = 0.0
    return Field(pos, np.full(n, a ** 3), nuc, m,
                 name=f"box_{nx}x{ny}x{nz}_a{a}" + ("_pores" if pores else ""))


def _rsa_centres(radii, cube, rng, max_tries=200):
    """Random sequential placement of non-overlapping spheres in a cube."""
    n = len(radii)
    centres = np.zeros((n, 3))
    cell = 2.0 * radii.max()
    grid = {}
    order = np.argsort(-radii)
    for idx in order:
        r = radii[idx]
        for _ in range(max_tries):
            c = rng.uniform(-cube / 2 + r, cube / 2 - r, size=3)
            key = tuple(np.floor(c / cell).astype(int))
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for j in grid.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                            if np.sum((centres[j] - c) ** 2) < (radii[j] + r) ** 2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                centres[idx] = c
                grid.setdefault(key, []).append(idx)
                break
        else:
            raise RuntimeError("could not place sphere without overlap")
    return centres


def sphere_ensemble(n_spheres=10000, median=8.0, sigma=0.35, clip=(5.0, 20.0), a=1.0,
                    cube=2000.0, canting=0.5, seed=3):
    """Ragged ensemble of spheres on their own local simple-cubic lattices.

    Radii lognormal(ln median, sigma) clipped to ``clip``; centres random,
    non-overlapping in a cube of side ``cube``.  Each sphere has a random easy
    axis e_k and a Neel-surface-like profile m = normalise(e_k + canting
    (r/R)^4 r_perp), r_perp the part of the unit radius vector normal to e_k.
    N_j = 1.  Cells are local coordinates; ``centers`` carry the positions.
    """
    rng = np.random.default_rng(seed)
    radii = np.clip(np.exp(np.log(median) + sigma * rng.normal(size=n_spheres)), clip[0], clip[1])
    centres = _rsa_centres(radii, cube, rng)
    axes = rng.normal(size=(n_spheres, 3))
    axes /= np.linalg.norm(axes, axis=1, keepdims=True)
    # sphere templates are cached by the radius quantised to the lattice
    cache = {}
    pos_l, mag_l, off = [], [], [0]
    for k in range(n_spheres):
        R = radii[k]
        key = round(R / a, 6)
        if key not in cache:
            cache[key] = lattice_ball(R, a)
        p = cache[key]
        rn = np.linalg.norm(p, axis=1)
        safe = np.where(rn > 0, rn, 1.0)
        u = p / safe[:, None]
        e = axes[k]
        uperp = u - (u @ e)[:, None] * e[None, :]
        m = e[None, :] + canting * (rn / R)[:, None] ** 4 * uperp
        pos_l.append(p)
        mag_l.append(_normalise(m))
        off.append(off[-1] + p.shape[0])
    pos = np.concatenate(pos_l)
    mag = np.concatenate(mag_l)
    n = pos.shape[0]
    return Field(pos, np.full(n, a ** 3), np.ones(n), mag, offsets=np.array(off),
                 centers=centres, name=f"ensemble_{n_spheres}")


def ellipsoid_uniform(semi=(40.0, 25.0, 25.0), a=0.8, seed=4):
    """Uniformly magnetised ellipsoid; m at a seeded polar angle to e_z."""
    rng = np.random.default_rng(seed)
    sa = np.asarray(semi, dtype=np.float64)
    m_ = np.floor(sa / a).astype(int) + 1
    gx = np.arange(-m_[0], m_[0] + 1) * a
    gy = np.arange(-m_[1], m_[1] + 1) * a
    gz = np.arange(-m_[2], m_[2] + 1) * a
    X, Y, Z = np.meshgrid(gx, gy, gz, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    keep = ((p / sa[None, :]) ** 2).sum(1) <= 1.0
    pos = p[keep]
    th = rng.uniform(0.0, np.pi / 2)
    ph = rng.uniform(0.0, 2 * np.pi)
    mdir = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    n = pos.shape[0]
    return Field(pos, np.full(n, a ** 3), np.ones(n), np.tile(mdir, (n, 1)), name="ellipsoid")


def random_rotations(n, seed=5):
    """n uniform random rotation matrices, row-major [n,3,3] (Shoemake's method)."""
    rng = np.random.default_rng(seed)
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    q = np.stack([np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
                  np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3),
                  np.sqrt(u1) * np.cos(2 * np.pi * u3)], axis=1)
    x, y, z, w = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


VORTEX_FAMILY_BOUNDS = np.array([
    [10.0, 40.0],   # particle radius (nm)
    [2.0, 8.0],     # core radius (nm)
    [-1.0, 1.0],    # chirality (sign taken)
    [-1.0, 1.0],    # polarity (sign taken)
    [0.0, 60.0],    # field canting angle (deg)
    [0.0, 2.0],     # N/M contrast
])


def vortex_family_params(n, seed=6):
    """n parameter rows [radius, core, chirality, polarity, canting_deg, contrast]."""
    rng = np.random.default_rng(seed)
    lo, hi = VORTEX_FAMILY_BOUNDS[:, 0], VORTEX_FAMILY_BOUNDS[:, 1]
    p = lo + (hi - lo) * rng.random((n, 6))
    p[:, 2] = np.where(p[:, 2] < 0, -1.0, 1.0)
    p[:, 3] = np.where(p[:, 3] < 0, -1.0, 1.0)
    return p


def vortex_family_member(params, a=2.0):
    """Vortex particle for one parameter row: curl of chirality c, Gaussian
    core of polarity p, the whole texture canted by the field angle about x,
    nuclear density equal to the contrast."""
    R, core, c, p, cant_deg, contrast = [float(v) for v in params]
    pos = lattice_ball(R, a)
    x, y = pos[:, 0], pos[:, 1]
    rho = np.hypot(x, y)
    safe = np.where(rho > 0, rho, 1.0)
    m = np.zeros_like(pos)
    m[:, 0] = np.where(rho > 0, -c * y / safe, 0.0)
    m[:, 1] = np.where(rho > 0, c * x / safe, 0.0)
    m[:, 2] = p * np.exp(-rho ** 2 / (2.0 * core * core))
    m = _normalise(m)
    t = np.deg2rad(cant_deg)
    ct, st = np.cos(t), np.sin(t)
    m = np.stack([m[:, 0], ct * m[:, 1] - st * m[:, 2], st * m[:, 1] + ct * m[:, 2]], axis=1)
    n = pos.shape[0]
    return Field(pos, np.full(n, a ** 3), np.full(n, contrast), m, name="vortex_member")


def replicate(field, copies):
    """The runtime-experiment shape: ``copies`` identical objects, dilute."""
    n = field.n
    pos = np.tile(field.pos, (copies, 1))
    vol = np.tile(field.vol, copies)
    nuc = None if field.nuc is None else np.tile(field.nuc, copies)
    mag = None if field.mag is None else np.tile(field.mag, (copies, 1))
    off = np.arange(copies + 1, dtype=np.int64) * n
    return Field(pos, vol, nuc, mag, offsets=off, centers=np.zeros((copies, 3)),
                 name=f"{field.name}_x{copies}")


def small_random_field(n_cells, seed=7, extent=10.0, n_objects=1):
    """Tiny random field for brute-force checks (positions uniform in a cube)."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-extent, extent, size=(n_cells, 3))
    vol = rng.uniform(0.5, 1.5, size=n_cells)
    nuc = rng.normal(size=n_cells)
    mag = rng.normal(size=(n_cells, 3))
    off = None
    cen = None
    if n_objects > 1:
        cuts = np.sort(rng.choice(np.arange(1, n_cells), size=n_objects - 1, replace=False))
        off = np.concatenate([[0], cuts, [n_cells]]).astype(np.int64)
        cen = rng.uniform(-3 * extent, 3 * extent, size=(n_objects, 3))
    return Field(pos, vol, nuc, mag, offsets=off, centers=cen, name="small_random")


def field_sweep(field, h_values, axis=(0.0, 0.0, 1.0)):
    """Magnetization states of one geometry along an applied-field sweep (loop
    mode input): state s is normalise(m + h_s * axis) per cell, with the
    field's own m as the zero-field state (cells with |m| = 0 stay 0).
    Returns (nuc [S][n], mag [S][n][3]); N is the same in every state."""
    m = np.asarray(field.mag, dtype=np.float64)
    ax = np.asarray(axis, dtype=np.float64)
    ax = ax / np.linalg.norm(ax)
    norm0 = np.linalg.norm(m, axis=1, keepdims=True)
    live = norm0 > 0
    mags = []
    for h in h_values:
        v = m + h * ax[None, :] * live
        nv = np.linalg.norm(v, axis=1, keepdims=True)
        mags.append(np.where(nv > 0, v / np.where(nv > 0, nv, 1.0) * norm0, 0.0))
    S = len(h_values)
    nuc = np.tile(field.nuc, (S, 1)) if field.nuc is not None else None
    return nuc, np.ascontiguousarray(np.stack(mags))
