"""Pins of the oracle's refinement-map rebuild (Sec. 2.1 step 4; readings
R21-R23).

* flag masks against an independent numpy statement of the criteria
  (density / pressure gradient across one cell, density threshold) and of
  the flag buffer, on random and on tanh-front data;
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


def numpy_masks(u, npg, criterion, thr, nb, bc=("periodic",) * 3):
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


def test_single_precision_flags_on_single_values():
    # the float evaluation decides like the double one away from ties
    u, npg = wl.lognormal_cells(32, seed=23, sigma=0.1)
    u32 = u.astype(np.float32).astype(np.float64)
    O = oracle.OracleLevels(wl.uniform_hierarchy(npg), [hm.domain_to_patches(u32, npg)])
    for crit, thr in ((0, 0.3), (1, 0.048), (2, 1.35)):
        a = O.flag_level(0, G, crit, thr, 2, single=True)
        b = O.flag_level(0, G, crit, thr, 2, single=False)
        assert np.mean(a == b) > 0.95


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
