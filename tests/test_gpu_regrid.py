"""The refinement-map rebuild on the GPU (Sec. 2.1 step 4; readings R21-R23)
against the oracle:

* flag masks: FP64 handles bit for bit against the oracle's double
  decision; FP32 handles against the same double decision, where a cell
  whose criterion lies within the oracle's bound on the single-precision
  rounding error of the threshold may go either way (the masks must lie
  between those of the cells flagged whatever the rounding and those of the
  cells that may be flagged; outside such ties they are equal bit for bit,
  and ties are rare); three criteria, three buffer sizes, one to three
  levels;
* refinement fill: FP64 bit for bit, FP32 within 1e-6 relative;
* a whole rebuild through paper_0907_3390_gb300.regrid against
  oracle.regrid, whose maps the oracle builds itself: the same levels and,
  element by element, the same group coordinates, parents, child maps and
  26-neighbour maps, and, in FP64, the same data bit for bit (FP32 inputs
  are checked to have no tie cell first), on periodic domains and on a
  tube with outflow ends;
* a blast evolved on the GPU with a rebuild every few pairs: the finest
  level follows the shock and the composite sums stay conserved.
"""
import sys
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import regrid as org  # noqa: E402
from paper_0907_3390_gb300 import binding as B  # noqa: E402
from paper_0907_3390_gb300 import hierarchy as hm  # noqa: E402
from paper_0907_3390_gb300 import regrid as rg  # noqa: E402
from paper_0907_3390_gb300 import workloads as wl  # noqa: E402

sys.path.insert(0, os.path.dirname(__file__))
from test_oracle_regrid import blast_two_level  # noqa: E402

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0
PREC = {"f32": (B.GAMER_FP32, torch.float32, np.float32), "f64": (B.GAMER_FP64, torch.float64, np.float64)}


def three_level():
    def score(level, centres):
        x, y, z = (centres[a][:, 0, 0, 0] for a in range(3))
        r = np.sqrt((x - 0.45) ** 2 + (y - 0.55) ** 2 + (z - 0.5) ** 2)
        return 0.3 - r if level == 0 else 0.17 - r
    H = hm.build_hierarchy((3, 3, 3), score, 3)

    def prim(x, y, z, dh):
        rho = 1.0 + 0.5 * np.tanh((x - 0.45) / 0.02) + 0.6 + 0.1 * np.sin(6 * np.pi * y)
        P = 1.0 + 0.8 * np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / 0.003)
        zr = np.zeros_like(x)
        return rho, zr + 0.1, zr, zr, P
    return H, wl.level_fields(H, prim)


def cases():
    u, npg = wl.lognormal_cells(32, seed=21, sigma=0.1)
    yield "one level", wl.single_level(u, npg), [(0, 0.3), (1, 0.048), (2, 1.35)]
    yield "blast", blast_two_level(), [(1, 0.5), (0, 0.01), (2, 1.0)]
    yield "three levels", three_level(), [(0, 0.05), (1, 0.05), (2, 1.5)]


U32 = 2.0 ** -24     # unit roundoff of single precision


def check_masks(got, O, l, crit, thr, nb, prec, stats=None):
    """FP64: the oracle's double decision bit for bit.  FP32: between the
    masks of the cells flagged whatever the single-precision rounding and
    those that may be flagged (equal where no tie cell contributes)."""
    if prec == "f64":
        want = O.flag_level(l, G, crit, thr, nb)
        assert np.array_equal(got, want)
        return
    sure, maybe, near = O.flag_level_bounds(l, G, crit, thr, nb, U32)
    assert not np.any(got & ~maybe), "a cell flagged that the double decision cannot flag"
    assert not np.any(sure & ~got), "a cell the double decision flags whatever the rounding is not flagged"
    if stats is not None:
        stats.append((near, 4096 * O.H.levels[l].n_groups))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_flag_masks_against_double_decision(prec):
    p, dt_, npdt = PREC[prec]
    stats = []
    for name, (H, st), crits in cases():
        S = B.Solver(G, 0, p)
        D = B.DeviceHierarchy(H, st, dt_)
        O = oracle.OracleLevels(H, [np.asarray(s).astype(npdt).astype(np.float64) for s in st])
        for crit, thr in crits:
            for nb in (0, 3, 8):
                for l in range(H.n_levels):
                    m = torch.full((8 * H.levels[l].n_groups,), -1, dtype=torch.int32, device="cuda")
                    B.gamer_hydro_flag(S.h, D, l, crit, thr, nb, m)
                    got = m.cpu().numpy().view(np.uint32)
                    check_masks(got, O, l, crit, thr, nb, prec, stats)
        S.close()
    if prec == "f32":
        near = sum(a for a, _ in stats)
        cells = sum(b for _, b in stats)
        assert near <= 1e-4 * cells, (near, cells)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_flag_threshold_at_representable_boundary(prec):
    """Thresholds equal to the largest criterion value and one double away on
    either side: the kernel compares in the handle's precision against
    thresholds rounded on the host, and must decide as the oracle, which
    widens the value to double (R21)."""
    p, dt_, npdt = PREC[prec]
    u, npg = wl.lognormal_cells(32, seed=21, sigma=0.1)
    H, st = wl.single_level(u, npg)
    S = B.Solver(G, 0, p)
    D = B.DeviceHierarchy(H, st, dt_)
    O = oracle.OracleLevels(H, [np.asarray(x).astype(npdt).astype(np.float64) for x in st])
    rho = u[0].astype(npdt)
    # largest relative density change over one cell width, periodic domain,
    # in the handle's precision and in the order of the criterion
    two = npdt(2)
    gmax = max(float(np.max(np.abs(np.roll(rho, -1, a) - np.roll(rho, 1, a)) / (two * np.abs(rho))))
               for a in range(3))
    m = torch.empty(8 * H.levels[0].n_groups, dtype=torch.int32, device="cuda")
    n_flagged = {}
    for crit, top in ((0, gmax), (2, float(rho.max()))):
        for name, thr in (("below", np.nextafter(top, -np.inf)), ("at", top), ("above", np.nextafter(top, np.inf))):
            B.gamer_hydro_flag(S.h, D, 0, crit, thr, 0, m)
            got = m.cpu().numpy().view(np.uint32)
            check_masks(got, O, 0, crit, thr, 0, prec)
            n_flagged[(crit, name)] = int(np.count_nonzero(got))
    # the boundary cases are the ones that decide: >= for the gradient, > for the threshold
    assert n_flagged[(0, "below")] >= 1 and n_flagged[(0, "at")] >= 1 and n_flagged[(0, "above")] == 0
    assert n_flagged[(2, "below")] >= 1 and n_flagged[(2, "at")] == 0 and n_flagged[(2, "above")] == 0
    S.close()


def outflow_tube():
    """A density front near the left end of a tube with outflow ends along x
    (periodic across), refined around the front: refined patches touch the
    outflow face, so rebuilt maps carry -2 entries."""
    def score(level, centres):
        x = centres[0][:, 0, 0, 0]
        return 0.2 - np.abs(x - 0.1) if level == 0 else -np.ones_like(x)
    H = hm.build_hierarchy((8, 1, 1), score, 2, bc=("outflow", "periodic", "periodic"))

    def prim(x, y, z, dh):
        rho = 1.0 + 0.6 * np.tanh((x - 0.06) / 0.01)
        zr = np.zeros_like(x)
        return rho, zr + 0.05, zr, zr, zr + 1.0
    return H, wl.level_fields(H, prim)


def rebuild_cases():
    yield from list(cases())[1:]
    yield "outflow tube", outflow_tube(), [(0, 0.05)]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_rebuild_matches_oracle(prec):
    p, dt_, npdt = PREC[prec]
    n_out = 0
    for name, (H, st), crits in rebuild_cases():
        crit, thr = crits[0]
        st_in = [np.asarray(s).astype(npdt).astype(np.float64) for s in st]
        if prec == "f32":
            # the double decision is the single-precision one on these inputs
            O = oracle.OracleLevels(H, st_in)
            for l in range(min(H.n_levels, 2)):
                assert O.flag_level_bounds(l, G, crit, thr, 2, U32)[2] == 0, (name, l)
        Ho, so = org.regrid(H, st_in, G, crit, [thr] * 3, 2, max_levels=3)
        S = B.Solver(G, 0, p)
        D = B.DeviceHierarchy(H, st, dt_)
        Dn = rg.rebuild(S, D, crit, [thr] * 3, 2, max_levels=3)
        assert Dn.H.n_levels == Ho.n_levels, name
        for l in range(Ho.n_levels):
            a, b = Dn.H.levels[l], Ho.levels[l]
            assert a.n_groups == b.n_groups, (name, l)
            assert np.array_equal(np.asarray(a.coords), np.asarray(b.coords)), (name, l)
            assert np.array_equal(np.asarray(a.nbr), np.asarray(b.nbr)), (name, l)
            n_out += int(np.count_nonzero(np.asarray(b.nbr) == -2)) if l > 0 else 0
            if l > 0:
                assert np.array_equal(a.parent, b.parent), (name, l)
            if l + 1 < Ho.n_levels:
                assert np.array_equal(a.child, b.child), (name, l)
            else:
                assert a.child is None or np.all(np.asarray(a.child) < 0), (name, l)
            got = Dn.u[l].double().cpu().numpy()
            if prec == "f64":
                assert np.array_equal(got, so[l]), (name, l)
            else:
                scale = np.abs(so[l]).reshape(5, -1).max(1)[:, None] + 1e-30
                assert (np.abs(got - so[l]).reshape(5, -1) / scale).max() <= 1e-6, (name, l)
        S.close()
    assert n_out > 0      # the outflow case reached the domain face


def test_blast_follows_refinement_and_conserves():
    H, st = blast_two_level()
    S = B.Solver(G, 0, B.GAMER_FP64)
    D = B.DeviceHierarchy(H, st, torch.float64)
    # one pair first so that covered coarse cells are restrictions
    B.gamer_hydro_step_pair(S.h, D, 0.4)
    s0, _ = B.gamer_hydro_check(S.h, D)
    for k in range(4):
        D = rg.rebuild(S, D, B.GAMER_FLAG_PRESSURE_GRADIENT, [0.3, 0.3], 2, max_levels=2)
        s1, nb = B.gamer_hydro_check(S.h, D)
        assert nb == 0
        assert np.all(np.abs(s1 - s0) / (np.abs(s0) + 1e-3) < 1e-12), (k, s1 - s0)
        for _ in range(2):
            B.gamer_hydro_step_pair(S.h, D, 0.4)
        s0, _ = B.gamer_hydro_check(S.h, D)
    # every level-0 patch that still sees a steep pressure gradient is refined
    m = torch.empty(8 * D.H.levels[0].n_groups, dtype=torch.int32, device="cuda")
    B.gamer_hydro_flag(S.h, D, 0, B.GAMER_FLAG_PRESSURE_GRADIENT, 0.6, 0, m)
    hit = np.nonzero(m.cpu().numpy())[0]
    assert len(hit) > 0
    child = D.H.levels[0].child
    assert np.mean(child[hit] >= 0) > 0.9
    S.close()
