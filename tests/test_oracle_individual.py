"""Pins of the oracle's individual time steps (Sec. 2.1: the time step of
level l may be half that of level l-1), readings R18-R20: a level's coarse
ghosts are interpolated in time between the coarser level's state before
and after its sweep set, and the coarser fix-up averages the finer fluxes
over the finer level's two steps.

* uniform flow stays bit-identical on three levels;
* composite sums over leaf cells are conserved to round-off on a periodic
  three-level hierarchy (catches any wrong flux weight or time level);
* a fully refined level evolves exactly like a single fine level with half
  the time step (no coarse ghosts, so the subcycling alone is tested), and
  the coarse level becomes the 8-cell means;
* time-interpolated coarse ghosts reproduce (u_old + u_new)/2 exactly on
  data linear in space;
* Eq. CFL for level 0 with individual steps is cfl min_l 2^l dh_l / s_l;
* on a smooth flow the result stays close to uniform time steps.
"""
import numpy as np
import pytest

import oracle
from paper_0907_3390_gb300 import hierarchy as hm
from paper_0907_3390_gb300 import workloads as wl

G = 5.0 / 3.0


def three_level():
    def score(level, centres):
        x, y, z = (centres[a][:, 0, 0, 0] for a in range(3))
        r = np.sqrt((x - 0.45) ** 2 + (y - 0.55) ** 2 + (z - 0.5) ** 2)
        return 0.3 - r if level == 0 else 0.17 - r
    H = hm.build_hierarchy((3, 3, 3), score, 3)
    assert H.n_levels == 3 and all(c > 0 for c in H.patch_counts())
    return H


def smooth_prim(x, y, z, dh):
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.1 * np.sin(2 * np.pi * z)
    vx = 0.3 * np.cos(2 * np.pi * y)
    vy = 0.2 * np.sin(2 * np.pi * z)
    vz = -0.25 * np.cos(2 * np.pi * x)
    P = 0.8 + 0.1 * np.cos(2 * np.pi * (x + y))
    return rho, vx, vy, vz, P


def test_uniform_flow_bitwise_individual():
    H = three_level()
    u = lambda x, y, z, dh: (np.full(x.shape, 1.25), np.full(x.shape, 0.5), np.full(x.shape, -0.75),
                             np.full(x.shape, 0.25), np.full(x.shape, 0.875))
    states = wl.level_fields(H, u)
    O = oracle.OracleLevels(H, states)
    for _ in range(2):
        O.cycle_individual(G, O.cfl_dt(G, 0.5, individual=True))
    for l in range(3):
        assert np.array_equal(O.u[l], states[l]), l


@pytest.mark.parametrize("lim", [oracle.VANLEER, oracle.MINMOD])
def test_composite_conservation_individual(lim):
    H = three_level()
    states = wl.level_fields(H, smooth_prim)
    O = oracle.OracleLevels(H, states)
    s0, _ = O.check(G)
    for _ in range(3):
        O.cycle_individual(G, O.cfl_dt(G, 0.5, individual=True), lim)
    s1, nb = O.check(G)
    assert nb == 0
    assert np.all(np.abs(s1 - s0) / (np.abs(s0) + 1e-3) < 1e-12), (s1 - s0)


def test_fully_refined_level_individual():
    def score(level, centres):
        return np.ones(centres.shape[1]) if level == 0 else np.zeros(centres.shape[1])
    H = hm.build_hierarchy((1, 1, 1), score, 2)
    assert H.patch_counts() == [8, 64]
    states = wl.level_fields(H, smooth_prim)
    O = oracle.OracleLevels(H, states)
    dt0 = O.cfl_dt(G, 0.5, individual=True)
    f = H.levels[1]
    fine_dom = np.empty((5, 32, 32, 32))
    for g in range(f.n_groups):
        cx, cy, cz = f.coords[g]
        fine_dom[:, 16 * cz:16 * cz + 16, 16 * cy:16 * cy + 16, 16 * cx:16 * cx + 16] = \
            hm.patches_to_domain(states[1][:, 8 * g:8 * g + 8], (1, 1, 1))
    Of = oracle.OracleLevels(wl.uniform_hierarchy((2, 2, 2)), [hm.domain_to_patches(fine_dom, (2, 2, 2))])
    O.cycle_individual(G, dt0)
    for order in (0, 1, 0, 1):                    # the fine level's four steps of dt0 / 2
        Of.step(G, 0.5 * dt0, order)
    fd = hm.patches_to_domain(Of.u[0], (2, 2, 2))
    for g in range(f.n_groups):
        cx, cy, cz = f.coords[g]
        blk = hm.patches_to_domain(O.u[1][:, 8 * g:8 * g + 8], (1, 1, 1))
        assert np.array_equal(blk, fd[:, 16 * cz:16 * cz + 16, 16 * cy:16 * cy + 16, 16 * cx:16 * cx + 16])
    coarse = hm.patches_to_domain(O.u[0], (1, 1, 1))
    avg = fd.reshape(5, 16, 2, 16, 2, 16, 2).sum(axis=(2, 4, 6))
    assert np.allclose(coarse, 0.125 * avg, rtol=1e-14, atol=0)


def test_time_interpolated_ghosts_linear():
    # fine groups inside a 4^3-group base, away from the edges
    def score(level, centres):
        if level > 0:
            return np.zeros(centres.shape[1])
        pc = np.floor(centres[:, :, 0, 0, 0] * 8).astype(int)     # patch coordinates (8 per unit)
        inside = np.ones(centres.shape[1], dtype=bool)
        for a, (lo, hi) in enumerate([(2, 4), (3, 5), (2, 4)]):
            inside &= (pc[a] >= lo) & (pc[a] < hi)
        return inside.astype(float) - 0.5
    H = hm.build_hierarchy((4, 4, 4), score, 2)
    assert H.patch_counts()[1] > 0
    aA, aB = np.array([0.25, -0.5, 0.75]), np.array([0.5, 0.25, -0.25])

    def field(a, c0):
        def prim(x, y, z, dh):
            r = c0 + a[0] * x + a[1] * y + a[2] * z
            zr = np.zeros_like(x)
            return r, zr + 0.125, zr, zr, r * 0 + 1.0
        return prim
    A = wl.level_fields(H, field(aA, 5.0))
    Bst = wl.level_fields(H, field(aB, 4.0))
    O = oracle.OracleLevels(H, A)
    O.flux2 = [[np.zeros((lv.n_groups, 3, 3, 5, 16, 16)) for _ in range(2)] for lv in H.levels]
    O.u_out[0][:] = Bst[0]                  # the coarse level's state after its sweep set
    O._cw[1] = 0.5
    f = H.levels[1]
    dh = f.dh
    am, cm = 0.5 * (aA + aB), 4.5
    idx = (np.arange(22) - 3 + 0.5) * dh
    n_ghost = 0
    for g in range(f.n_groups):
        blk = O.gather_block(1, g)
        lo = f.coords[g] * 16 * dh
        zz, yy, xx = np.meshgrid(lo[2] + idx, lo[1] + idx, lo[0] + idx, indexing="ij")
        exact = cm + am[0] * xx + am[1] * yy + am[2] * zz
        own = np.zeros((22, 22, 22), dtype=bool)
        own[3:19, 3:19, 3:19] = True
        # interior: this level's own (time-t) data; ghosts from coarse: mean of old and new
        nbr_fine = np.zeros((22, 22, 22), dtype=bool)
        for d, (dx, dy, dz) in enumerate(hm.DIRS):
            if f.nbr[g, hm.dir_index(dx, dy, dz)] >= 0:
                sl = [slice(3 + 16 * 0, 19)] * 3
                for ax, o in zip((2, 1, 0), (dx, dy, dz)):
                    sl[ax] = slice(0, 3) if o < 0 else (slice(19, 22) if o > 0 else slice(3, 19))
                nbr_fine[tuple(sl)] = True
        coarse_ghost = ~own & ~nbr_fine
        n_ghost += coarse_ghost.sum()
        assert np.allclose(blk[0][coarse_ghost], exact[coarse_ghost], rtol=0, atol=1e-13)
    assert n_ghost > 0


def test_cfl_individual_closed_form():
    H = three_level()
    O = oracle.OracleLevels(H, wl.level_fields(H, smooth_prim))
    s = [O.max_speed(l, G) for l in range(3)]
    want = 0.5 * min(2 ** l * H.levels[l].dh / s[l] for l in range(3))
    assert O.cfl_dt(G, 0.5, individual=True) == pytest.approx(want, rel=1e-15)
    assert O.cfl_dt(G, 0.5) == pytest.approx(0.5 * min(H.levels[l].dh / s[l] for l in range(3)), rel=1e-15)


def test_individual_close_to_uniform_on_smooth_flow():
    H = three_level()
    states = wl.level_fields(H, smooth_prim)
    Oi = oracle.OracleLevels(H, states)
    Ou = oracle.OracleLevels(H, states)
    dt0 = 0.5 * Oi.cfl_dt(G, 0.5, individual=True)
    Oi.cycle_individual(G, dt0)
    # uniform steps over the same time: every level takes dt0 / 4 eight times
    for k in range(8):
        Ou.step(G, dt0 / 4, k % 2)
    for l in range(3):
        d = np.abs(Oi.u[l] - Ou.u[l]).reshape(5, -1).max(1) / np.abs(Ou.u[l]).reshape(5, -1).max(1)
        assert d.max() < 2e-3, (l, d)
