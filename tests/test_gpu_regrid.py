"""The refinement-map rebuild on the GPU (Sec. 2.1 step 4; readings R21-R23)
against the oracle:

* flag masks bit for bit (the criteria are evaluated in the handle's
  precision on both sides: for an FP32 handle the oracle takes the same
  FP32 values and decides in single precision), three criteria and three
  buffer sizes, on one, two and three levels;
* refinement fill: FP64 bit for bit, FP32 within 1e-6 relative;
* a whole rebuild through paper_0907_3390_gb300.regrid against
  oracle.regrid: the same levels, groups, parents and, in FP64, the same
  data bit for bit;
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


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_flag_masks_bitwise(prec):
    p, dt_, npdt = PREC[prec]
    for name, (H, st), crits in cases():
        S = B.Solver(G, 0, p)
        D = B.DeviceHierarchy(H, st, dt_)
        O = oracle.OracleLevels(H, [np.asarray(s).astype(npdt).astype(np.float64) for s in st])
        for crit, thr in crits:
            for nb in (0, 3, 8):
                for l in range(H.n_levels):
                    m = torch.empty(8 * H.levels[l].n_groups, dtype=torch.int32, device="cuda")
                    B.gamer_hydro_flag(S.h, D, l, crit, thr, nb, m)
                    got = m.cpu().numpy().view(np.uint32)
                    want = O.flag_level(l, G, crit, thr, nb, single=prec == "f32")
                    assert np.array_equal(got, want), (name, crit, nb, l)
        S.close()


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
            want = O.flag_level(0, G, crit, thr, 0, single=prec == "f32")
            assert np.array_equal(got, want), (crit, name)
            n_flagged[(crit, name)] = int(np.count_nonzero(got))
    # the boundary cases are the ones that decide: >= for the gradient, > for the threshold
    assert n_flagged[(0, "below")] >= 1 and n_flagged[(0, "at")] >= 1 and n_flagged[(0, "above")] == 0
    assert n_flagged[(2, "below")] >= 1 and n_flagged[(2, "at")] == 0 and n_flagged[(2, "above")] == 0
    S.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_rebuild_matches_oracle(prec):
    p, dt_, npdt = PREC[prec]
    for name, (H, st), crits in list(cases())[1:]:
        crit, thr = crits[0]
        st_in = [np.asarray(s).astype(npdt).astype(np.float64) for s in st]
        Ho, so = org.regrid(H, st_in, G, crit, [thr] * 3, 2, max_levels=3, single=prec == "f32")
        S = B.Solver(G, 0, p)
        D = B.DeviceHierarchy(H, st, dt_)
        Dn = rg.rebuild(S, D, crit, [thr] * 3, 2, max_levels=3)
        assert Dn.H.n_levels == Ho.n_levels, name
        for l in range(Ho.n_levels):
            assert np.array_equal(np.asarray(Dn.H.levels[l].coords), np.asarray(Ho.levels[l].coords)), (name, l)
            if l > 0:
                assert np.array_equal(Dn.H.levels[l].parent, Ho.levels[l].parent), (name, l)
                assert np.array_equal(Dn.H.levels[l].nbr, Ho.levels[l].nbr), (name, l)
            got = Dn.u[l].double().cpu().numpy()
            if prec == "f64":
                assert np.array_equal(got, so[l]), (name, l)
            else:
                scale = np.abs(so[l]).reshape(5, -1).max(1)[:, None] + 1e-30
                assert (np.abs(got - so[l]).reshape(5, -1) / scale).max() <= 1e-6, (name, l)
        S.close()


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
