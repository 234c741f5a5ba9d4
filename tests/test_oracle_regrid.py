"""Pins of the oracle's refinement-map rebuild (Sec. 2.1 step 4; readings
R21-R23).

* flag masks against an independent numpy statement of the criteria
  (density / pressure gradient across one cell, density threshold) and of
  the flag buffer, on random and on tanh-front data;
* the bound on the criterion's rounding error in single precision: every
  float32 evaluation (three operation orders) lies within it, it is not
  vacuous, and float masks at exact ties lie between the sure and the
  possible masks;
* buffer closed forms: n_buffer = 0 flags only the patch itself, n_buffer
  = 8 every sibling;
* refinement fill: Min-Mod children conserve the parent cell and reproduce
  linear data exactly, inherited groups are copied bit for bit;
* the rules: a patch with a flagged child stays refined, a patch whose
  26 neighbours are not all on its level is not refined, and the cells that
  satisfy the criterion end up refined;
* composite sums over leaf cells are unchanged by a rebuild that follows a
  step (the coarse data under fine patches are then restrictions).
"""
import numpy as np
import pytest

import oracle
from oracle import regrid as org
from paper_0907_3390_gb300 import hierarchy as hm
from paper_0907_3390_gb300 import workloads as wl

G = 5.0 / 3.0


def numpy_masks(u, npg, criterion, thr, nb, bc=("periodic",) * 3, r_override=None):
    """Independent statement of the flag step on a single level given as a
    domain array u[5][nz][ny][nx]."""
    rho = u[0]
    if criterion == 1:
        v2 = (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / rho
        q = (G - 1.0) * (u[4] - 0.5 * v2)
        # the oracle's pressure uses v = m / rho; recompute it that way
        vx, vy, vz = u[1] / rho, u[2] / rho, u[3] / rho
        q = (G - 1.0) * (u[4] - 0.5 * rho * (vx * vx + vy * vy + vz * vz))
    else:
        q = rho
    if criterion == 2:
        hit = rho > thr
    elif r_override is not None:
        hit = r_override >= thr
    else:
        r = np.zeros_like(q)
        for ax in range(3):
            a = 2 - ax                      # array axis of x, y, z
            if bc[ax] == "periodic":
                qp, qm = np.roll(q, -1, a), np.roll(q, 1, a)
            else:
                pad = [(0, 0)] * 3
                pad[a] = (1, 1)
                qq = np.pad(q, pad, mode="edge")
                sl_p = [slice(None)] * 3
                sl_m = [slice(None)] * 3
                sl_p[a] = slice(2, None)
                sl_m[a] = slice(0, -2)
                qp, qm = qq[tuple(sl_p)], qq[tuple(sl_m)]
            r = np.maximum(r, np.abs(qp - qm) / (2.0 * np.abs(q)))
        hit = r >= thr
    nz, ny, nx = q.shape
    ppx, ppy, ppz = nx // 8, ny // 8, nz // 8
    masks = {}
    for z, y, x in zip(*np.nonzero(hit)):
        k = (x // 8, y // 8, z // 8)
        c = (x % 8, y % 8, z % 8)
        rng = [range(-1 if c[a] - nb < 0 else 0, (1 if c[a] + nb > 7 else 0) + 1) for a in range(3)]
        for dz in rng[2]:
            for dy in rng[1]:
                for dx in rng[0]:
                    masks[k] = masks.get(k, 0) | (1 << ((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)))
    out = np.zeros(8 * npg[0] * npg[1] * npg[2], dtype=np.uint32)
    H = wl.uniform_hierarchy(npg, bc=bc)
    coords = org._patch_coords(H.levels[0])
    for p, k in coords.items():
        out[p] = masks.get(k, 0)
    return H, out


@pytest.mark.parametrize("criterion,thr", [(0, 0.3), (1, 0.048), (2, 1.35)])
@pytest.mark.parametrize("nb", [0, 3, 8])
def test_flag_masks_against_numpy(criterion, thr, nb):
    u, npg = wl.lognormal_cells(32, seed=21, sigma=0.1)
    H, want = numpy_masks(u, npg, criterion, thr, nb)
    O = oracle.OracleLevels(H, [hm.domain_to_patches(u, npg)])
    got = O.flag_level(0, G, criterion, thr, nb)
    assert np.array_equal(got, want)
    assert got.any() and not np.all(got == got[0])


def test_flag_masks_outflow_front():
    # a density front along x in an outflow tube: gradient cells and their buffers
    u, npg, bc = wl.sod(0, 64, 16)
    H, want = numpy_masks(u, npg, 0, 0.03, 4, bc=bc)
    O = oracle.OracleLevels(H, [hm.domain_to_patches(u, npg)])
    got = O.flag_level(0, G, 0, 0.03, 4)
    assert np.array_equal(got, want)
    assert np.count_nonzero(got) > 0


U32 = 2.0 ** -24     # unit roundoff of single precision


def f32_criterion(u, criterion, order):
    """The criterion of every cell of a periodic domain u[5][nz][ny][nx]
    (values already single-precision numbers) evaluated in numpy float32,
    with one of several operation orders, all algebraically the same."""
    f = np.float32
    w = [np.asarray(x, dtype=f) for x in u]
    rho = w[0]
    if criterion == 0:
        q = rho
    else:
        gm1 = f(G - 1.0)
        if order == 0:
            vx, vy, vz = w[1] / rho, w[2] / rho, w[3] / rho
            q = gm1 * (w[4] - f(0.5) * rho * (vx * vx + vy * vy + vz * vz))
        elif order == 1:
            vx, vy, vz = w[1] / rho, w[2] / rho, w[3] / rho
            q = (w[4] - (f(0.5) * rho) * ((vz * vz + vy * vy) + vx * vx)) * gm1
        else:
            vx, vy, vz = w[1] / rho, w[2] / rho, w[3] / rho
            q = gm1 * (w[4] - f(0.5) * (w[1] * vx + w[2] * vy + w[3] * vz))
    n = np.zeros_like(q)
    for a in range(3):
        n = np.maximum(n, np.abs(np.roll(q, -1, a) - np.roll(q, 1, a)))
    with np.errstate(divide="ignore", invalid="ignore"):
        r = n / (f(2) * np.abs(q))
    return np.where(r > 0, r, f(0)).astype(np.float64)


@pytest.mark.parametrize("criterion", [0, 1])
def test_flag_error_bound_holds_for_float_evaluations(criterion):
    """The oracle's bound on the criterion's rounding error at unit
    roundoff u contains every single-precision evaluation, in three
    operation orders, on rough data (lognormal density, velocities up to
    a few times the sound speed, so that the pressure loses digits to
    cancellation), and is tight to within two orders of magnitude."""
    for seed, sigma in ((31, 0.5), (32, 1.5)):
        u, npg = wl.lognormal_cells(32, seed=seed, sigma=sigma)
        u[1:4] *= 3.0                    # faster flows: kinetic energy dominates e
        u[4] += 0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / u[0] * (1 - 1 / 9.0)
        u32 = u.astype(np.float32).astype(np.float64)
        O = oracle.OracleLevels(wl.uniform_hierarchy(npg), [hm.domain_to_patches(u32, npg)])
        val, bound = O.flag_criterion(0, G, criterion, U32)
        r64 = hm.patches_to_domain(val[None], npg)[0]
        b = hm.patches_to_domain(bound[None], npg)[0]
        ok = np.isfinite(b)
        assert ok.mean() > 0.999
        worst = 0.0
        for order in (0, 1, 2) if criterion == 1 else (0,):
            r32 = f32_criterion(u32, criterion, order)
            err = np.abs(r32 - r64)
            assert np.all(err[ok] <= b[ok]), (order, np.max(err[ok] / b[ok]))
            worst = max(worst, float(np.max(err[ok] / np.maximum(b[ok], 1e-300))))
        assert worst > 0.01, worst       # the bound is not vacuous


def test_flag_bounds_contain_float_masks_at_ties():
    """Thresholds placed exactly at single-precision criterion values (the
    hardest ties): the masks of a float evaluation lie between the masks of
    the cells flagged whatever the rounding and those that may be flagged,
    the double decision too; only the tie cells may differ."""
    u, npg = wl.lognormal_cells(32, seed=33, sigma=0.5)
    u32 = u.astype(np.float32).astype(np.float64)
    H = wl.uniform_hierarchy(npg)
    O = oracle.OracleLevels(H, [hm.domain_to_patches(u32, npg)])
    for crit in (0, 1):
        r32 = f32_criterion(u32, crit, 0)
        for thr in np.sort(r32.ravel())[-3:-400:-97]:
            sure, maybe, near = O.flag_level_bounds(0, G, crit, float(thr), 1, U32)
            exact = O.flag_level(0, G, crit, float(thr), 1)
            _, m32 = numpy_masks(u32, npg, crit, float(thr), 1, r_override=r32)
            for m in (m32, exact):
                assert not np.any(m & ~maybe) and not np.any(sure & ~m)
            assert near >= 1 and near < 50
            s0, m0, n0 = O.flag_level_bounds(0, G, crit, float(thr), 1, 0.0)
            assert np.array_equal(s0, exact) and np.array_equal(m0, exact) and n0 == 0


def test_flag_density_threshold_has_no_ties():
    # the density criterion compares a stored value: no rounding, no tie band
    u, npg = wl.lognormal_cells(32, seed=34, sigma=0.5)
    u32 = u.astype(np.float32).astype(np.float64)
    O = oracle.OracleLevels(wl.uniform_hierarchy(npg), [hm.domain_to_patches(u32, npg)])
    thr = float(np.sort(u32[0].ravel())[-50])
    sure, maybe, near = O.flag_level_bounds(0, G, 2, thr, 0, U32)
    assert near == 0 and np.array_equal(sure, maybe)
    assert np.array_equal(sure, O.flag_level(0, G, 2, thr, 0))


def test_buffer_closed_forms():
    u, npg = wl.lognormal_cells(32, seed=22, sigma=0.3)
    O = oracle.OracleLevels(wl.uniform_hierarchy(npg), [hm.domain_to_patches(u, npg)])
    m0 = O.flag_level(0, G, 2, 1.0, 0)
    assert np.all((m0 == 0) | (m0 == 1 << 13))
    m8 = O.flag_level(0, G, 2, 1.0, 8)
    assert np.all((m8 == 0) | (m8 == (1 << 27) - 1))
    assert np.array_equal(m0 != 0, m8 != 0)


def two_level_linear():
    def score(level, centres):
        if level > 0:
            return np.zeros(centres.shape[1])
        pc = np.floor(centres[:, :, 0, 0, 0] * 8).astype(int)
        inside = np.ones(centres.shape[1], dtype=bool)
        for a, (lo, hi) in enumerate([(2, 4), (3, 5), (2, 4)]):
            inside &= (pc[a] >= lo) & (pc[a] < hi)
        return inside.astype(float) - 0.5
    return hm.build_hierarchy((4, 4, 4), score, 2)


def test_refine_fill_linear_exact_conservative_and_inherit():
    H = two_level_linear()
    a = np.array([0.25, -0.5, 0.75])

    def lin(x, y, z, dh):
        r = 5.0 + a[0] * x + a[1] * y + a[2] * z
        zr = np.zeros_like(x)
        return r, zr + 0.125, zr, zr, r * 0 + 1.0
    st = wl.level_fields(H, lin)
    O = oracle.OracleLevels(wl.uniform_hierarchy((4, 4, 4)), [st[0]])
    f = H.levels[1]
    # new level: the same parents; group 0 inherits old group 1, the rest is interpolated
    inherit = np.full(f.n_groups, -1, dtype=np.int32)
    inherit[0] = 1
    Hc = hm.Hierarchy(levels=[H.levels[0]], base_npg=H.base_npg)
    Oc = oracle.OracleLevels(Hc, [st[0]], with_flux=False)
    out = Oc.refine_fill(0, f.parent, inherit, st[1])
    assert np.array_equal(out[:, 0:8], st[1][:, 8:16])
    # interpolated groups: exact on linear data (Min-Mod keeps the slope)
    cen = H.cell_centres(1)
    exact = 5.0 + a[0] * cen[0] + a[1] * cen[1] + a[2] * cen[2]
    assert np.allclose(out[0, 8:], exact[8:], rtol=0, atol=1e-13)
    # conservative: the 8 children of every coarse cell average to it
    for i in range(1, f.n_groups):
        P = f.parent[i]
        kids = hm.patches_to_domain(out[:, 8 * i:8 * i + 8], (1, 1, 1))      # [5][16][16][16]
        mean = kids.reshape(5, 8, 2, 8, 2, 8, 2).mean(axis=(2, 4, 6))
        coarse = st[0][:, P]                                                   # [5][8][8][8]
        assert np.allclose(mean, coarse, rtol=1e-14, atol=0)


def blast_two_level():
    # a 64^3 base with a small refined region away from the blast, Sedov-like
    # energy in the centre: the rebuild must move the fine level to the blast
    def score(level, centres):
        if level > 0:
            return np.zeros(centres.shape[1])
        pc = np.floor(centres[:, :, 0, 0, 0] * 8).astype(int)
        inside = np.ones(centres.shape[1], dtype=bool)
        for a, (lo, hi) in enumerate([(0, 2), (0, 2), (0, 2)]):
            inside &= (pc[a] >= lo) & (pc[a] < hi)
        return inside.astype(float) - 0.5
    H = hm.build_hierarchy((4, 4, 4), score, 2)

    def prim(x, y, z, dh):
        r2 = (x - 0.55) ** 2 + (y - 0.55) ** 2 + (z - 0.55) ** 2
        P = 1e-2 + np.exp(-r2 / 0.002)
        zr = np.zeros_like(x)
        return zr + 1.0, zr, zr, zr, P
    return H, wl.level_fields(H, prim)


def test_rebuild_rules_and_criterion_coverage():
    H, st = blast_two_level()
    thr = [0.5, 0.5, 0.5]
    Hn, sn = org.regrid(H, st, G, 1, thr, 2, max_levels=3)
    O = oracle.OracleLevels(H, st)
    # every level-0 cell that satisfies the criterion is now under a level-1 patch
    m0 = O.flag_level(0, G, 1, thr[0], 0)
    hit = {org._patch_coords(H.levels[0])[p] for p in np.nonzero(m0)[0]}
    f = Hn.levels[1]
    covered = {tuple(int(c) for c in f.coords[g]) for g in range(f.n_groups)}
    assert hit and hit <= covered
    # proper nesting of the result and consistent maps
    for l in range(Hn.n_levels):
        hm.validate_level(Hn.levels, l)
    for l in range(1, Hn.n_levels):
        lv = Hn.levels[l]
        par = Hn.levels[l - 1]
        pc = org._patch_coords(par)
        look = {v: k for k, v in pc.items()}
        ext = [2 * e for e in par.extent]
        for g in range(lv.n_groups):
            k = pc[int(lv.parent[g])]
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        assert ((k[0] + dx) % ext[0], (k[1] + dy) % ext[1], (k[2] + dz) % ext[2]) in look
    # the old refined corner is gone: nothing there satisfies the criterion
    assert (0, 0, 0) not in covered and (1, 1, 1) not in covered


def test_children_keep_their_parents_refined():
    # three levels; a threshold that only the finest level's cells exceed:
    # level 0 sees no cell above it, yet keeps the parent of the level-1
    # patch whose children stay
    def score(level, centres):
        x, y, z = (centres[a][:, 0, 0, 0] for a in range(3))
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        return 0.3 - r if level == 0 else 0.15 - r
    H = hm.build_hierarchy((4, 4, 4), score, 3)

    def prim(x, y, z, dh):
        r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
        rho = 1.0 + 3.0 * np.exp(-r2 / (2 * (1.5 * dh) ** 2)) * (dh < 0.01)
        zr = np.zeros_like(x)
        return rho, zr, zr, zr, zr + 1.0
    st = wl.level_fields(H, prim)
    O0 = oracle.OracleLevels(H, st)
    assert not O0.flag_level(0, G, 2, 1.5, 1).any()      # no level-0 cell above the threshold
    Hn, sn = org.regrid(H, st, G, 2, [1.5, 1.5, 1.5], 1, max_levels=3)
    assert Hn.n_levels == 3 and Hn.levels[1].n_groups > 0 and Hn.levels[2].n_groups > 0


def test_rebuild_after_a_step_conserves_composite_sums():
    H, st = blast_two_level()
    O = oracle.OracleLevels(H, st)
    dt = O.cfl_dt(G, 0.5)
    O.step(G, dt, 0)            # the fix-up makes covered coarse cells restrictions
    s0, _ = O.check(G)
    Hn, sn = org.regrid(H, O.u, G, 1, [0.5, 0.5, 0.5], 2, max_levels=3)
    On = oracle.OracleLevels(Hn, sn)
    s1, _ = On.check(G)
    assert np.all(np.abs(s1 - s0) / (np.abs(s0) + 1e-3) < 1e-12), (s1 - s0)


def _geometry_nbr(fine, bc):
    """Neighbour map of a level from its group coordinates alone: the group
    at coords + d (wrapped on periodic axes), -2 past an outflow face, -1
    where no group of the level sits."""
    ext = fine.extent
    pos = {tuple(int(v) for v in fine.coords[g]): g for g in range(fine.n_groups)}
    out = np.empty((fine.n_groups, 26), dtype=np.int32)
    for g in range(fine.n_groups):
        k = [int(v) for v in fine.coords[g]]
        j = 0
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if (dx, dy, dz) == (0, 0, 0):
                        continue
                    q = [k[0] + dx, k[1] + dy, k[2] + dz]
                    val = None
                    for a in range(3):
                        if q[a] < 0 or q[a] >= ext[a]:
                            if bc[a] == "periodic":
                                q[a] %= ext[a]
                            else:
                                val = -2
                    out[g, j] = val if val is not None else pos.get(tuple(q), -1)
                    j += 1
    return out


@pytest.mark.parametrize("bc", [("periodic",) * 3, ("outflow", "periodic", "outflow")])
def test_refine_maps_against_geometry(bc):
    """The oracle's rebuilt maps (a walk through the coarse neighbour map)
    against the geometry of the group coordinates, over random sets of
    properly nested patches on two successive levels."""
    rng = np.random.default_rng(5)
    H = wl.uniform_hierarchy((3, 2, 3), bc=bc)
    cur = org._own_level(H.levels[0])
    for lev in range(2):
        pc = org.patch_coords(cur)
        nested = [p for p in range(8 * cur.n_groups) if org.properly_nested(cur, p)]
        assert nested
        refine = sorted(rng.choice(nested, size=max(1, len(nested) // 2), replace=False).tolist())
        fine, child = org.refine_maps(cur, refine)
        assert np.array_equal(fine.nbr, _geometry_nbr(fine, bc))
        for i, p in enumerate(refine):
            assert tuple(int(v) for v in fine.coords[i]) == pc[p]
            assert child[p] == i and fine.parent[i] == p
        assert np.count_nonzero(child >= 0) == len(refine)
        if bc[0] == "outflow":
            assert np.any(fine.nbr == -2)
        cur = fine
    # a patch next to an unrefined region of the coarser level is not nested
    assert not all(org.properly_nested(cur, p) for p in range(8 * cur.n_groups))
