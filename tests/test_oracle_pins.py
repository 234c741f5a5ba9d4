"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, exact symmetries of the scheme, invariants (conservation, uniform
flow), brute-force tables, or a structurally different formulation.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_0907_3390_gb300 import hierarchy as hm
from paper_0907_3390_gb300 import workloads as wl

G = 5.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- limiters

VALS = [-3.0, -1.0, -0.25, 0.0, 0.5, 1.0, 2.0, 7.0]


def test_vanleer_table():
    """Eq. vanLeer: zero unless both corrections share a sign; otherwise the
    harmonic mean 2/(1/a + 1/b), symmetric, odd, bounded by 2 min(|a|,|b|)."""
    for a, b in itertools.product(VALS, VALS):
        p = oracle.phi_vanleer(a, b)
        if a * b <= 0:
            assert p == 0.0
        else:
            assert p == pytest.approx(2.0 / (1.0 / a + 1.0 / b), rel=1e-15)
            assert abs(p) <= 2 * min(abs(a), abs(b)) + 1e-15
            assert np.sign(p) == np.sign(a)
        assert oracle.phi_vanleer(b, a) == p
        assert oracle.phi_vanleer(-a, -b) == -p
    assert oracle.phi_vanleer(1.5, 1.5) == 1.5


def test_vanleer_tvd_region():
    """Sweby form phi(r) = 2r/(1+r) of van Leer (a = 1, b = r) for r > 0."""
    for r in np.linspace(0.01, 20.0, 97):
        assert oracle.phi_vanleer(1.0, r) == pytest.approx(2 * r / (1 + r), rel=1e-14)


def test_minmod_table():
    for a, b in itertools.product(VALS, VALS):
        p = oracle.phi_minmod(a, b)
        if a * b <= 0:
            assert p == 0.0
        else:
            assert abs(p) == min(abs(a), abs(b)) and np.sign(p) == np.sign(a)
        assert oracle.phi_minmod(b, a) == p


# ------------------------------------------------------------------ EOS

def test_pressure_roundtrip():
    """Eqs. ThermalEnergy + EOS: P recovered from e = P/(g-1) + rho v^2/2."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        rho, P = rng.uniform(0.1, 10), rng.uniform(0.01, 10)
        v = rng.normal(0, 2, 3)
        u = wl.prim_to_cons(np.array(rho), *[np.array(x) for x in v], np.array(P))
        assert oracle.pressure(u, G) == pytest.approx(P, rel=1e-12)


# ------------------------------------------------------------- 1-D column

def _rand_column(rng, L=22):
    rho = rng.uniform(0.5, 2.0, L)
    v = rng.normal(0, 0.5, (3, L))
    P = rng.uniform(0.5, 2.0, L)
    return wl.prim_to_cons(rho, v[0], v[1], v[2], P).T.copy()


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("lim", [oracle.VANLEER, oracle.MINMOD])
def test_column_mirror_symmetry(d, lim):
    """Reflecting the column (x -> -x, v_d -> -v_d) reflects the result
    bit for bit: the left-moving TVD flux mirrors the right-moving one
    (reading R4)."""
    rng = np.random.default_rng(11 + d)
    q = _rand_column(rng)
    out = oracle.tvd_column(q, d, 0.2, G, lim)
    qm = q[::-1].copy()
    qm[:, 1 + d] *= -1
    om = oracle.tvd_column(qm, d, 0.2, G, lim)
    om = om[::-1].copy()
    om[:, 1 + d] *= -1
    assert np.array_equal(out[3:19], om[3:19])


def test_column_uniform_exact():
    q = np.tile(wl.prim_to_cons(np.array(1.3), np.array(0.4), np.array(-0.2), np.array(0.1),
                                np.array(0.8)), (22, 1))
    for d in range(3):
        assert np.array_equal(oracle.tvd_column(q, d, 0.3, G)[3:19], q[3:19])


def test_column_zero_dt_identity():
    rng = np.random.default_rng(3)
    q = _rand_column(rng)
    assert np.array_equal(oracle.tvd_column(q, 0, 0.0, G), q)


def test_column_local_stencil():
    """Seven-point stencil (Sec. 2.2): perturbing cell m changes only cells
    m-3..m+3 of the result."""
    rng = np.random.default_rng(8)
    q = _rand_column(rng, 30)
    base = oracle.tvd_column(q, 0, 0.2, G)
    for m in (8, 14, 20):
        q2 = q.copy()
        q2[m, 0] *= 1.01
        o2 = oracle.tvd_column(q2, 0, 0.2, G)
        changed = np.nonzero(np.any(o2[3:27] != base[3:27], axis=1))[0] + 3
        assert changed.min() >= m - 3 and changed.max() <= m + 3
        assert m in changed


def test_column_first_order_limit_upwind_advection():
    """Linear advection check of the flux splitting: a passive density
    contrast at uniform v, P is carried downwind (mass moves toward +x for
    v > 0) and the total mass of the column is conserved with the boundary
    fluxes of a constant state."""
    L = 40
    rho = np.where(np.arange(L) < 20, 2.0, 1.0)
    z = np.zeros(L)
    q = wl.prim_to_cons(rho, z + 0.5, z, z, z + 1.0).T.copy()
    o = oracle.tvd_column(q, 0, 0.1, G)
    # the jump moves right: cell 20 gains mass, cell 19 does not grow
    assert o[20, 0] > q[20, 0]
    assert o[19, 0] <= q[19, 0] + 1e-15
    # away from the jump nothing changes
    assert np.array_equal(o[3:14], q[3:14]) and np.array_equal(o[27:37], q[27:37])


# ---------------------------------------------------------- whole domain

def _conserved_drift(u0, u1):
    s0 = u0.reshape(5, -1).sum(1)
    s1 = u1.reshape(5, -1).sum(1)
    scale = np.abs(u0).reshape(5, -1).sum(1)
    return np.abs(s1 - s0) / scale


@pytest.mark.parametrize("lim", [oracle.VANLEER, oracle.MINMOD])
def test_uniform_flow_preserved_bitwise(lim):
    u, npg = wl.uniform_flow(16)
    for order in (0, 1):
        out = oracle.domain_sweepset(u, G, 0.01, 1 / 16, order, lim)
        assert np.array_equal(out, u)
    H, st = wl.single_level(u, npg)
    O = oracle.OracleLevels(H, st)
    oracle.run(O, G, 0.5, 4, lim)
    assert np.array_equal(O.u[0], st[0])


def test_periodic_conservation_roundoff():
    """The flux form telescopes on a periodic domain: the totals of the five
    conserved variables drift only by round-off over 20 sweep sets."""
    u, npg = wl.lognormal_cells(32, seed=1000)
    H, st = wl.single_level(u, npg)
    O = oracle.OracleLevels(H, st)
    oracle.run(O, G, 0.5, 20)
    d = _conserved_drift(st[0], O.u[0])
    assert np.all(d < 1e-13), d


def test_domain_equals_patch_groups_bitwise():
    """Two formulations: domain-wide split sweeps vs padded patch groups with
    ghost zones (Sec. 3.1) give identical results on one level, for both
    sweep orders, periodic and outflow boundaries."""
    u, npg = wl.lognormal_cells(32, seed=1000)
    dh = 1.0 / 32
    H, st = wl.single_level(u, npg)
    O = oracle.OracleLevels(H, st)
    dt = 0.4 * O.cfl_dt(G, 1.0)
    ud = u.copy()
    for order in (0, 1, 0):
        ud = oracle.domain_sweepset(ud, G, dt, dh, order)
        O.step(G, dt, order)
    assert np.array_equal(hm.patches_to_domain(O.u[0], npg), ud)
    us, npg2, bc = wl.sod(0, 64, 16)
    H2, st2 = wl.single_level(us, npg2, bc=bc)
    O2 = oracle.OracleLevels(H2, st2)
    ud2 = us.copy()
    dt = 0.4 * O2.cfl_dt(G, 1.0)
    for order in (0, 1):
        ud2 = oracle.domain_sweepset(ud2, G, dt, H2.levels[0].dh, order, bc=bc)
        O2.step(G, dt, order)
    assert np.array_equal(hm.patches_to_domain(O2.u[0], npg2), ud2)


def test_sod_direction_symmetry_bitwise():
    """A 1-D problem run along x, y and z gives bit-identical profiles:
    transverse sweeps are exact identities when transverse momenta vanish."""
    prof = []
    for ax in range(3):
        u, npg, bc = wl.sod(ax, 128, 16)
        H, st = wl.single_level(u, npg, bc=bc)
        O = oracle.OracleLevels(H, st)
        oracle.run(O, G, 0.5, 20)
        d = hm.patches_to_domain(O.u[0], npg)
        # move the tube axis to the last position and take one line
        d = np.moveaxis(d, 3 - ax, 3)
        line = d[:, 5, 7, :].copy()
        # the normal momentum sits in slot 1+ax
        mom = line[1 + ax].copy()
        others = [line[1 + a] for a in range(3) if a != ax]
        assert all(np.all(o == 0.0) for o in others)
        prof.append(np.stack([line[0], mom, line[4]]))
        # every transverse line is identical
        assert np.all(d == d[:, :1, :1, :])
    assert np.array_equal(prof[0], prof[1]) and np.array_equal(prof[0], prof[2])


def test_domain_mirror_symmetry_3d():
    """x -> -x reflection of a random 3-D state commutes with one sweep set."""
    u, npg = wl.lognormal_cells(16, seed=77)
    out = oracle.domain_sweepset(u, G, 0.002, 1 / 16, 0)
    um = u[:, :, :, ::-1].copy()
    um[1] *= -1
    om = oracle.domain_sweepset(um, G, 0.002, 1 / 16, 0)[:, :, :, ::-1].copy()
    om[1] *= -1
    assert np.array_equal(out, om)


# ---------------------------------------------------- Min-Mod prolongation

def test_minmod_children_conservative_and_linear_exact():
    rng = np.random.default_rng(2)
    for _ in range(20):
        blk = rng.uniform(0.5, 2.0, (5, 3, 3, 3))
        ch = oracle.minmod_children(blk)
        assert np.allclose(ch.reshape(5, -1).mean(1), blk[:, 1, 1, 1], rtol=0, atol=1e-15)
    # linear data: exact values at child centres (offsets +-1/4 cell)
    a, b, c, d0 = 0.3, -0.2, 0.15, 2.0
    k, j, i = np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij")
    blk = np.stack([d0 + a * i + b * j + c * k] * 5)
    ch = oracle.minmod_children(blk)
    kk, jj, ii = np.meshgrid([-0.25, 0.25], [-0.25, 0.25], [-0.25, 0.25], indexing="ij")
    assert np.allclose(ch[0], d0 + a * ii + b * jj + c * kk, atol=1e-15)
    # a local extremum has zero slope: all children equal the parent
    blk = np.ones((5, 3, 3, 3))
    blk[:, 1, 1, 1] = 3.0
    assert np.all(oracle.minmod_children(blk) == 3.0)


# -------------------------------------------------------------- hierarchy

def two_level(n0=2, box=None, fields=None, seed=4):
    """A periodic (16 n0)^3 base with the patches in ``box`` (patch coords,
    inclusive-exclusive per axis) refined."""
    def score(level, centres):
        if level > 0:
            return np.zeros(centres.shape[1])
        pc = np.floor(centres[:, :, 0, 0, 0] / (8 * (1.0 / (16 * n0)))).astype(int)  # [3, 8n]
        inside = np.ones(centres.shape[1], dtype=bool)
        for a in range(3):
            inside &= (pc[a] >= box[a][0]) & (pc[a] < box[a][1])
        return inside.astype(float) - 0.5
    H = hm.build_hierarchy((n0, n0, n0), score, 2)
    return H


def _smooth_prim(x, y, z, dh):
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.1 * np.sin(2 * np.pi * z)
    vx = 0.3 * np.cos(2 * np.pi * y)
    vy = 0.2 * np.sin(2 * np.pi * z)
    vz = -0.25 * np.cos(2 * np.pi * x)
    P = 0.8 + 0.1 * np.cos(2 * np.pi * (x + y))
    return rho, vx, vy, vz, P


def test_proper_nesting_and_maps():
    H = two_level(2, box=[(1, 3), (1, 3), (1, 3)])
    assert H.patch_counts() == [64, 64]
    for l in range(2):
        hm.validate_level(H.levels, l)
    f = H.levels[1]
    pos = {tuple(c): g for g, c in enumerate(f.coords)}
    for g in range(f.n_groups):
        for (dx, dy, dz) in hm.DIRS:
            q = tuple((f.coords[g] + (dx, dy, dz)) % 8)
            want = pos.get(q, -1)
            assert f.nbr[g, hm.dir_index(dx, dy, dz)] == want
    # every fine group has exactly 7 fine neighbours (a 2x2x2 block of groups)
    assert np.all((f.nbr >= 0).sum(1) == 7)
    # parents are the refined patches, and child inverts parent
    c = H.levels[0].child
    for g in range(f.n_groups):
        assert c[f.parent[g]] == g
    assert (c >= 0).sum() == f.n_groups


def test_fully_refined_equals_fine_single_level():
    """If every coarse patch is refined, the fine level sees no coarse
    ghosts: it must evolve exactly like a single level at fine resolution,
    and the coarse level must become the 8-cell average (restriction)."""
    def score(level, centres):
        return np.ones(centres.shape[1]) if level == 0 else np.zeros(centres.shape[1])
    H = hm.build_hierarchy((1, 1, 1), score, 2)
    assert H.patch_counts() == [8, 64]
    states = wl.level_fields(H, _smooth_prim)
    O = oracle.OracleLevels(H, states)
    dt = 0.3 * O.cfl_dt(G, 1.0)
    # single fine level with the same data
    Hf = wl.uniform_hierarchy((2, 2, 2))
    fine_dom = np.empty((5, 32, 32, 32))
    # place each fine group by its coordinates
    f = H.levels[1]
    for g in range(f.n_groups):
        cx, cy, cz = f.coords[g]
        blk = hm.patches_to_domain(states[1][:, 8 * g:8 * g + 8], (1, 1, 1))
        fine_dom[:, 16 * cz:16 * cz + 16, 16 * cy:16 * cy + 16, 16 * cx:16 * cx + 16] = blk
    Of = oracle.OracleLevels(Hf, [hm.domain_to_patches(fine_dom, (2, 2, 2))])
    for order in (0, 1):
        O.step(G, dt, order)
        Of.step(G, dt, order)
    fd = hm.patches_to_domain(Of.u[0], (2, 2, 2))
    for g in range(f.n_groups):
        cx, cy, cz = f.coords[g]
        blk = hm.patches_to_domain(O.u[1][:, 8 * g:8 * g + 8], (1, 1, 1))
        assert np.array_equal(blk, fd[:, 16 * cz:16 * cz + 16, 16 * cy:16 * cy + 16, 16 * cx:16 * cx + 16])
    coarse = hm.patches_to_domain(O.u[0], (1, 1, 1))
    avg = fd.reshape(5, 16, 2, 16, 2, 16, 2)
    avg = ((((((avg[:, :, 0, :, 0, :, 0] + avg[:, :, 0, :, 0, :, 1]) + avg[:, :, 0, :, 1, :, 0]) +
               avg[:, :, 0, :, 1, :, 1]) + avg[:, :, 1, :, 0, :, 0]) + avg[:, :, 1, :, 0, :, 1]) +
            avg[:, :, 1, :, 1, :, 0]) + avg[:, :, 1, :, 1, :, 1]
    assert np.allclose(coarse, 0.125 * avg, rtol=1e-15, atol=0)


def test_coarse_ghosts_exact_on_linear_data():
    """Ghost cells interpolated from the coarser level (Sec. 2.2) reproduce a
    linear field exactly at the fine cell centres when no slope is clipped."""
    H = two_level(4, box=[(2, 4), (3, 5), (2, 4)])
    a = np.array([0.3, -0.5, 0.7])

    def lin(x, y, z, dh):
        r = 5.0 + a[0] * x + a[1] * y + a[2] * z
        zr = np.zeros_like(x)
        return r, zr + 0.1, zr, zr, r * 0 + 1.0
    states = wl.level_fields(H, lin)
    O = oracle.OracleLevels(H, states)
    f = H.levels[1]
    dh = f.dh
    for g in range(f.n_groups):
        blk = O.gather_block(1, g)
        lo = f.coords[g] * 16 * dh
        idx = (np.arange(22) - 3 + 0.5) * dh
        zz, yy, xx = np.meshgrid(lo[2] + idx, lo[1] + idx, lo[0] + idx, indexing="ij")
        exact = 5.0 + a[0] * xx + a[1] * yy + a[2] * zz
        assert np.allclose(blk[0], exact, rtol=0, atol=1e-13)
        assert np.allclose(blk[1], 0.1 * exact, rtol=0, atol=1e-13)


def test_amr_uniform_flow_bitwise():
    H = two_level(2, box=[(1, 3), (0, 2), (1, 3)])
    # dyadic values: the 8-child sums of the restriction are exact
    u = lambda x, y, z, dh: (np.full(x.shape, 1.25), np.full(x.shape, 0.5), np.full(x.shape, -0.75),
                             np.full(x.shape, 0.25), np.full(x.shape, 0.875))
    states = wl.level_fields(H, u)
    O = oracle.OracleLevels(H, states)
    oracle.run(O, G, 0.5, 4)
    for l in range(2):
        assert np.array_equal(O.u[l], states[l])


def _composite_sums(O):
    sums, _ = O.check(G)
    return sums


@pytest.mark.parametrize("lim", [oracle.VANLEER, oracle.MINMOD])
def test_amr_composite_conservation(lim):
    """Restriction + Berger-Colella flux correction (Sec. 2.1, step 3) keep
    the composite totals over leaf cells constant to round-off on a periodic
    three-level hierarchy."""
    def score(level, centres):
        x, y, z = (centres[a][:, 0, 0, 0] for a in range(3))
        r = np.sqrt((x - 0.45) ** 2 + (y - 0.55) ** 2 + (z - 0.5) ** 2)
        return 0.3 - r if level == 0 else 0.17 - r
    H = hm.build_hierarchy((3, 3, 3), score, 3)
    assert H.n_levels == 3 and all(c > 0 for c in H.patch_counts())
    states = wl.level_fields(H, _smooth_prim)
    O = oracle.OracleLevels(H, states)
    s0 = _composite_sums(O)
    scale = np.abs(s0) + 1e-3
    oracle.run(O, G, 0.5, 6, lim)
    s1 = _composite_sums(O)
    assert np.all(np.abs(s1 - s0) / scale < 1e-12), (s1 - s0) / scale


# ------------------------------------------------------------ CFL / check

def test_cfl_closed_form():
    """Eq. CFL: uniform rho = 1, P = 3/5 (c_s = 1), v = (0.5, -2, 0.1): the
    signal speed is 1 + 2 = 3 and dt = cfl * dh / 3."""
    s = (32, 32, 32)
    u = wl.prim_to_cons(np.ones(s), np.full(s, 0.5), np.full(s, -2.0), np.full(s, 0.1), np.full(s, 0.6))
    H, st = wl.single_level(u, (2, 2, 2))
    O = oracle.OracleLevels(H, st)
    assert O.cfl_dt(G, 0.5) == pytest.approx(0.5 * (1 / 32) / 3.0, rel=1e-14)


def test_cfl_multilevel_min():
    H = two_level(2, box=[(1, 3), (1, 3), (1, 3)])
    speeds = {0: 1.0, 1: 0.8}

    def st(l):
        n = 8 * H.levels[l].n_groups
        shp = (n, 8, 8, 8)
        vx = speeds[l] if l == 0 else speeds[l]
        return wl.prim_to_cons(np.ones(shp), np.full(shp, vx), np.zeros(shp), np.zeros(shp), np.full(shp, 0.6))
    O = oracle.OracleLevels(H, [st(0), st(1)])
    dh0 = H.levels[0].dh
    # level 0: dh0 / 2, level 1: (dh0/2) / 1.8
    assert O.cfl_dt(G, 1.0) == pytest.approx(min(dh0 / 2.0, 0.5 * dh0 / 1.8), rel=1e-14)


def test_check_sums_and_bad_cells():
    u, npg = wl.uniform_flow(32)
    H, st = wl.single_level(u, npg)
    O = oracle.OracleLevels(H, st)
    sums, nb = O.check(G)
    assert nb == 0
    assert np.allclose(sums, u[:, 0, 0, 0] * 1.0, rtol=1e-13)  # volume of the unit box
    bad = st[0].copy()
    bad[0, 3, 1, 2, 3] = -1.0           # negative density
    bad[4, 9, 0, 0, 0] = 0.0            # negative pressure
    bad[2, 20, 5, 5, 5] = np.nan        # non-finite
    O2 = oracle.OracleLevels(H, [bad])
    assert O2.check(G)[1] == 3


def test_check_skips_covered_cells():
    H = two_level(2, box=[(1, 3), (1, 3), (1, 3)])
    states = wl.level_fields(H, lambda x, y, z, dh: (np.ones(x.shape),) + (np.zeros(x.shape),) * 3 +
                             (np.full(x.shape, 0.6),))
    states[0][0, np.nonzero(H.levels[0].child >= 0)[0][0]] = -5.0   # covered: ignored
    O = oracle.OracleLevels(H, states)
    sums, nb = O.check(G)
    assert nb == 0
    assert sums[0] == pytest.approx(1.0, rel=1e-13)


def test_golden_file_citations():
    with open(os.path.join(GOLDEN, "paper_values.json")) as f:
        gold = json.load(f)
    for k, v in gold.items():
        assert "cite" in v and "value" in v, k
