"""Seeded synthetic inputs shaped like the paper's test problems and runs.

Everything here is input construction: random fields, initial conditions
and hierarchies.  None of the solver's arithmetic lives here; the only
physics used is the ideal-gas relation that turns primitive variables into
conserved ones, e = P/(gamma-1) + rho |v|^2 / 2 (Eqs. ThermalEnergy, EOS),
applied once to build the initial state that both the CUDA path and the CPU
oracle receive.

Seeds: NumPy PCG64, one seed per workload.  Fields are generated in FP64 on
the host; the FP32 path receives them cast once.

Workloads (sizes in cells; each 8^3 patch belongs to a 16^3 patch group):
* ``lognormal_cells``: periodic 32^3 (64 patches), cell-wise
  rho = exp(sigma g - sigma^2/2), g ~ N(0,1), sigma = 0.5 (E[rho] = 1),
  P = 1 + 0.1 U(0,1), v_i ~ N(0, 0.3).
* ``sod``: 128 x 16 x 16 tube along x, y or z; rho 1 / 0.125, P 1 / 0.1,
  v = 0, interface at the middle; outflow along the tube, periodic across
  (the shock-tube set-up of Sec. 4.2).
* ``smooth_grf``: periodic 128^3 (4096 patches), Gaussian random fields
  with P(k) ~ k^-2; rho = exp(a delta) with a chosen so max/min = 10,
  P = rho^gamma, three velocity fields scaled to rms Mach 1.
* ``lognormal_grf``: periodic 512^3 (262,144 patches) by default,
  rho = exp(sigma delta - sigma^2/2) with sigma = 1.5, P = 1, k^-2 velocity
  fields scaled to rms Mach 3.
* ``amr_grf``: a 128^3 base with two finer levels placed where a seeded
  lognormal k^-2 density exceeds per-level thresholds (about 4096 / 9000 /
  21000 patches), fields sampled at every level's cell centres.
* ``amr_stress``: four levels, about 32,768 patches: lognormal density with
  sigma 2.5 (contrast up to ~1e5) and converging flows up to Mach 20, or a
  Sedov point blast (E = 1 in one finest cell, rho = 1, P = 1e-5).
* ``acoustic_wave``: rho0 = 1, P0 = 3/5 (c_s = 1), standing sinusoidal
  density perturbation of relative amplitude 1e-6 along a diagonal, flow at
  rest (Sec. 4.1).
"""
from __future__ import annotations

import os

import numpy as np

from .hierarchy import (GROUP, PATCH, Hierarchy, LevelMap, build_hierarchy,
                        domain_to_patches, uniform_level)

GAMMA = 5.0 / 3.0


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def prim_to_cons(rho, vx, vy, vz, P, gamma=GAMMA) -> np.ndarray:
    """Conserved (rho, rho v, e) from primitives; e = P/(gamma-1) + rho v^2/2."""
    e = P / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return np.stack([rho, rho * vx, rho * vy, rho * vz, e])


# ------------------------------------------------------------ random fields

def grf(n: int, rng: np.random.Generator, index: float = -2.0) -> np.ndarray:
    """Periodic Gaussian random field on n^3 cells with P(k) ~ k^index,
    zero mean and unit variance (white noise shaped in Fourier space)."""
    white = rng.standard_normal((n, n, n))
    f = np.fft.rfftn(white)
    kx = np.fft.rfftfreq(n)[None, None, :]
    ky = np.fft.fftfreq(n)[None, :, None]
    kz = np.fft.fftfreq(n)[:, None, None]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (index / 2.0)
    d = np.fft.irfftn(f * amp, s=(n, n, n), axes=(0, 1, 2))
    d -= d.mean()
    d /= d.std()
    return d


def _sample_chunk(flat, n, fx, fy, fz):
    ix, iy, iz = np.floor(fx).astype(np.int64), np.floor(fy).astype(np.int64), np.floor(fz).astype(np.int64)
    tx, ty, tz = fx - ix, fy - iy, fz - iz
    xs = (ix % n, (ix + 1) % n)
    ys = (iy % n * n, (iy + 1) % n * n)
    zs = (iz % n * (n * n), (iz + 1) % n * (n * n))
    out = 0.0
    for dz in (0, 1):
        wz = tz if dz else 1.0 - tz
        for dy in (0, 1):
            wy = ty if dy else 1.0 - ty
            zy = zs[dz] + ys[dy]
            for dx in (0, 1):
                wx = tx if dx else 1.0 - tx
                out = out + wx * wy * wz * np.take(flat, zy + xs[dx])
    return out


def sample_periodic(field: np.ndarray, x, y, z, L: float = 1.0) -> np.ndarray:
    """Trilinear interpolation of a periodic cell-centred field [nz][ny][nx]
    at physical positions (x, y, z) in [0, L)^3 (input construction only).
    Large requests are split into chunks evaluated on a thread pool; every
    value is formed by the same operations in the same order either way."""
    n = field.shape[0]
    flat = np.ascontiguousarray(field).ravel()
    x, y, z = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64),
                                  np.asarray(z, dtype=np.float64))
    shape = x.shape
    fx = (x / L * n - 0.5).ravel()
    fy = (y / L * n - 0.5).ravel()
    fz = (z / L * n - 0.5).ravel()
    m = fx.size
    chunk = 1 << 20
    if m <= chunk:
        return np.asarray(_sample_chunk(flat, n, fx, fy, fz)).reshape(shape)
    import concurrent.futures as cf
    out = np.empty(m)

    def one(a):
        b = min(a + chunk, m)
        out[a:b] = _sample_chunk(flat, n, fx[a:b], fy[a:b], fz[a:b])
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(one, range(0, m, chunk)))
    return out.reshape(shape)


# ------------------------------------------------------ single-level inputs

def lognormal_cells(n: int = 32, seed: int = 1000, sigma: float = 0.5):
    """Cell-wise lognormal density, uniform-random pressure, Gaussian
    velocities on a periodic n^3 domain.  Returns (u[5][n][n][n], npg)."""
    rng = rng_for(seed)
    g = rng.standard_normal((n, n, n))
    rho = np.exp(sigma * g - 0.5 * sigma * sigma)
    P = 1.0 + 0.1 * rng.random((n, n, n))
    v = rng.normal(0.0, 0.3, (3, n, n, n))
    return prim_to_cons(rho, v[0], v[1], v[2], P), (n // GROUP,) * 3


def sod(axis: int = 0, n_long: int = 128, n_tr: int = 16):
    """Sod shock tube along ``axis`` (Sec. 4.2 initial state).  Returns
    (u[5][nz][ny][nx], npg, bc)."""
    shape = [n_tr, n_tr, n_tr]
    shape[2 - axis] = n_long
    shape = tuple(shape)
    idx = np.indices(shape)[2 - axis]
    left = idx < n_long // 2
    rho = np.where(left, 1.0, 0.125)
    P = np.where(left, 1.0, 0.1)
    z = np.zeros(shape)
    u = prim_to_cons(rho, z, z, z, P)
    npg = (shape[2] // GROUP, shape[1] // GROUP, shape[0] // GROUP)
    bc = ["periodic"] * 3
    bc[axis] = "outflow"
    return u, npg, tuple(bc)


def uniform_flow(n: int = 32, rho=1.3, v=(0.4, -0.7, 0.25), P=0.9):
    s = (n, n, n)
    return prim_to_cons(np.full(s, rho), np.full(s, v[0]), np.full(s, v[1]), np.full(s, v[2]),
                        np.full(s, P)), (n // GROUP,) * 3


def smooth_grf(n: int = 128, seed: int = 1001, contrast: float = 10.0, mach: float = 1.0,
               gamma: float = GAMMA):
    """k^-2 Gaussian random fields: density contrast ``contrast``,
    P = rho^gamma, rms Mach ``mach``.  Returns (u, npg)."""
    rng = rng_for(seed)
    d = grf(n, rng)
    a = np.log(contrast) / (d.max() - d.min())
    rho = np.exp(a * (d - d.mean()))
    P = rho ** gamma
    v = np.stack([grf(n, rng) for _ in range(3)])
    cs2 = gamma * P / rho
    s = mach / np.sqrt(np.mean((v * v).sum(0) / cs2))
    v *= s
    return prim_to_cons(rho, v[0], v[1], v[2], P, gamma), (n // GROUP,) * 3


def lognormal_grf(n: int = 512, seed: int = 1003, sigma: float = 1.5, mach: float = 3.0,
                  gamma: float = GAMMA, dtype=np.float64):
    """Lognormal k^-2 density (sigma in ln rho), P = 1, k^-2 velocities at
    rms Mach ``mach``.  Returns (u, npg)."""
    rng = rng_for(seed)
    d = grf(n, rng)
    rho = np.exp(sigma * d - 0.5 * sigma * sigma)
    del d
    P = np.ones_like(rho)
    v = np.stack([grf(n, rng) for _ in range(3)])
    cs2 = gamma * P / rho
    s = mach / np.sqrt(np.mean((v * v).sum(0) / cs2))
    v *= s
    u = prim_to_cons(rho, v[0], v[1], v[2], P, gamma)
    return u.astype(dtype, copy=False), (n // GROUP,) * 3


def acoustic_wave(n: int, amp: float = 1e-6, n_z: int | None = None):
    """Standing sound wave along the (1,1,0) diagonal of an n x n x n_z
    periodic box of unit side, one wavelength across the box diagonal
    period.  rho0 = 1, P0 = 3/5, gamma = 5/3 (c_s = 1), at rest.  Returns
    (u, k_vec, npg) where rho(x,t) = 1 + amp sin(k.x) cos(|k| t)."""
    n_z = n if n_z is None else n_z
    z, y, x = np.meshgrid((np.arange(n_z) + 0.5) / n, (np.arange(n) + 0.5) / n,
                          (np.arange(n) + 0.5) / n, indexing="ij")
    k = np.array([2 * np.pi, 2 * np.pi, 0.0])
    ph = k[0] * x + k[1] * y
    rho = 1.0 + amp * np.sin(ph)
    P = 0.6 + amp * np.sin(ph)   # c_s^2 drho with c_s = 1
    zr = np.zeros_like(rho)
    return prim_to_cons(rho, zr, zr, zr, P), k, (n // GROUP, n // GROUP, max(n_z // GROUP, 1))


# ------------------------------------------------------------ AMR inputs

def amr_hierarchy(base_npg, targets, density_sampler, L: float = 1.0) -> Hierarchy:
    """Hierarchy whose level l+1 holds ``targets[l+1]`` patches (when enough
    patches are eligible under proper nesting) placed where the patch
    maximum of ``density_sampler(x, y, z)`` is largest."""
    def score(level, centres):
        vals = density_sampler(centres[0], centres[1], centres[2])
        return vals.reshape(vals.shape[0], -1).max(axis=1)
    return build_hierarchy(base_npg, score, len(targets), targets=list(targets), L=L)


def level_fields(H: Hierarchy, prim_fn, gamma=GAMMA):
    """Conserved state of every level, prim_fn(x, y, z, dh) -> (rho, vx, vy,
    vz, P) evaluated at the level's cell centres."""
    out = []
    for l in range(H.n_levels):
        c = H.cell_centres(l)
        rho, vx, vy, vz, P = prim_fn(c[0], c[1], c[2], H.levels[l].dh)
        out.append(prim_to_cons(rho, vx, vy, vz, P, gamma))
    return out


def smoothed(field: np.ndarray, R: float) -> np.ndarray:
    """Gaussian smoothing (radius R cells) of a periodic field in Fourier space."""
    n = field.shape[0]
    k2 = (np.fft.rfftfreq(n)[None, None, :] ** 2 + np.fft.fftfreq(n)[None, :, None] ** 2 +
          np.fft.fftfreq(n)[:, None, None] ** 2) * (2 * np.pi) ** 2
    return np.fft.irfftn(np.fft.rfftn(field) * np.exp(-0.5 * k2 * R * R), s=field.shape, axes=(0, 1, 2))


def amr_grf(seed: int = 1002, base_n: int = 128, targets=(4096, 9000, 21000), n_field: int = 128,
            sigma: float = 1.0, mach: float = 1.0, gamma: float = GAMMA):
    """Three-level hierarchy over a periodic base_n^3 grid; returns (H, [u_l]).

    Refinement is placed where the density smoothed over ~2 base patches is
    highest (compact regions, as flag buffers make them in the paper)."""
    rng = rng_for(seed)
    d = grf(n_field, rng)
    vf = [grf(n_field, rng) for _ in range(3)]
    sel = smoothed(d, 2.0 * PATCH * n_field / base_n)
    vscale = mach * np.sqrt(gamma)  # rms Mach ~ mach for rho ~ P ~ 1

    def dens(x, y, z):
        return np.exp(sigma * sample_periodic(d, x, y, z) - 0.5 * sigma * sigma)

    H = amr_hierarchy((base_n // GROUP,) * 3, list(targets),
                      lambda x, y, z: sample_periodic(sel, x, y, z))

    def prim(x, y, z, dh):
        rho = dens(x, y, z)
        P = rho ** gamma
        v = [vscale * sample_periodic(f, x, y, z) for f in vf]
        return rho, v[0], v[1], v[2], P
    return H, level_fields(H, prim, gamma)


def amr_stress(kind: str = "lognormal", seed: int = 1004, base_n: int = 64,
               targets=(512, 4096, 12288, 15872), n_field: int = 64, gamma: float = GAMMA):
    """Four-level stress hierarchy (about 32,768 patches in total).

    kind='lognormal': density exp(2.5 delta - 2.5^2/2) clipped to a 1e5
    contrast, converging velocities toward the density peaks scaled so the
    largest Mach number is 20, P = 1e-2 rho.
    kind='sedov': rho = 1, P = 1e-5, v = 0, E = 1 of thermal energy put in
    one finest-level cell at a seeded position."""
    rng = rng_for(seed)
    if kind == "lognormal":
        d = grf(n_field, rng)
        sig = 2.5
        lo, hi = -0.5 * np.log(1e5), 0.5 * np.log(1e5)

        def lnrho(x, y, z):
            return np.clip(sig * sample_periodic(d, x, y, z) - 0.5 * sig * sig, lo + 0.0, hi)

        gx, gy, gz = np.gradient(d, 1.0 / n_field)
        sel = smoothed(d, 2.0 * PATCH * n_field / base_n)
        H = amr_hierarchy((base_n // GROUP,) * 3, list(targets),
                          lambda x, y, z: sample_periodic(sel, x, y, z))
        vmax = 0.0
        gmax = np.sqrt(gx * gx + gy * gy + gz * gz).max()

        def prim(x, y, z, dh):
            rho = np.exp(lnrho(x, y, z))
            P = 1e-2 * rho
            cs = np.sqrt(gamma * P / rho)
            # flow along +grad(delta): converges on density peaks
            v = [sample_periodic(g, x, y, z) / gmax for g in (gx, gy, gz)]
            return rho, 20.0 * cs * v[0], 20.0 * cs * v[1], 20.0 * cs * v[2], P
        return H, level_fields(H, prim, gamma)
    if kind == "sedov":
        centre = rng.random(3)

        def dist(x, y, z):
            dd = 0.0
            for a, q in enumerate((x, y, z)):
                t = np.abs(q - centre[a])
                t = np.minimum(t, 1.0 - t)
                dd = dd + t * t
            return np.sqrt(dd)

        H = amr_hierarchy((base_n // GROUP,) * 3, list(targets), lambda x, y, z: -dist(x, y, z))
        # the finest cell containing the centre gets E = 1
        lf = H.n_levels - 1

        def prim(x, y, z, dh):
            s = x.shape
            rho = np.ones(s)
            P = np.full(s, 1e-5)
            zr = np.zeros(s)
            return rho, zr, zr, zr, P
        us = level_fields(H, prim, gamma)
        c = H.cell_centres(lf)
        dh = H.levels[lf].dh
        inside = np.all([np.abs(c[a] - centre[a]) <= 0.5 * dh for a in range(3)], axis=0)
        idx = np.argwhere(inside)
        if len(idx) == 0:   # the centre is not on the finest level: nearest cell
            dd = dist(c[0], c[1], c[2])
            idx = np.argwhere(dd == dd.min())[:1]
        p, k, j, i = idx[0]
        us[lf][4, p, k, j, i] += 1.0 / dh ** 3
        return H, us
    raise ValueError(kind)


def uniform_hierarchy(npg, L: float = 1.0, bc=("periodic",) * 3) -> Hierarchy:
    lv = uniform_level(npg, dh=L / (GROUP * npg[0]), bc=bc)
    return Hierarchy(levels=[lv], base_npg=tuple(npg), L=L)


def single_level(u_domain: np.ndarray, npg, L: float = 1.0, bc=("periodic",) * 3):
    """Hierarchy + patch-layout state of a one-level domain array."""
    H = uniform_hierarchy(npg, L=L, bc=bc)
    return H, [domain_to_patches(u_domain, npg)]


# ------------------------------------------------------------ potentials

def potential_blocks(phi_fn, npg, dh: float) -> np.ndarray:
    """[n_groups][18][18][18] potential blocks of a one-level domain of
    (nx, ny, nz) patch groups: phi_fn(x, y, z) evaluated at the cell centres
    of every group and of its one-cell ghost layer, x fastest, groups in the
    order g = (gz ny + gy) nx + gx.  phi_fn is any callable on arrays (an
    external potential or a test field)."""
    nx, ny, nz = npg
    i = np.arange(GROUP + 2, dtype=np.float64) - 0.5          # ghost centre at -0.5 dh
    out = np.empty((nx * ny * nz, GROUP + 2, GROUP + 2, GROUP + 2))
    for g in range(nx * ny * nz):
        gx, gy, gz = g % nx, (g // nx) % ny, g // (nx * ny)
        z, y, x = np.meshgrid((gz * GROUP + i) * dh, (gy * GROUP + i) * dh, (gx * GROUP + i) * dh, indexing="ij")
        out[g] = phi_fn(x, y, z)
    return out


def periodic_potential_blocks(phi: np.ndarray, npg) -> np.ndarray:
    """[n_groups][18][18][18] blocks cut from a periodic [nz][ny][nx] cell
    array (ghost layer wrapped), groups in the order g = (gz ny + gy) nx + gx."""
    nx, ny, nz = npg
    p = np.pad(phi, 1, mode="wrap")
    out = np.empty((nx * ny * nz, GROUP + 2, GROUP + 2, GROUP + 2), dtype=phi.dtype)
    for g in range(nx * ny * nz):
        gx, gy, gz = g % nx, (g // nx) % ny, g // (nx * ny)
        out[g] = p[gz * GROUP:gz * GROUP + GROUP + 2, gy * GROUP:gy * GROUP + GROUP + 2,
                   gx * GROUP:gx * GROUP + GROUP + 2]
    return out
