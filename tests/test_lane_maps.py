"""The thread-to-column tables of the FP32 sweeps (lane_maps.h): generated
from gen_lane_maps.py, each a permutation of its sweep's columns, and with
fewer shared-memory bank conflicts per warp than the natural order."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0907_3390_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_lane_maps", os.path.join(CSRC, "gen_lane_maps.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_header_is_generated():
    g = _gen()
    with open(os.path.join(CSRC, "lane_maps.h")) as f:
        assert f.read() == g.render()


def test_tables_are_permutations_with_fewer_conflicts():
    g = _gen()
    for name, order, s, perm, before, after, warps in g.tables():
        cols, bank = g.phase_columns(order, s)
        assert sorted(perm) == sorted(cols) and len(set(perm)) == len(cols), name
        assert all(0 <= i1 < g.PD and 0 <= i2 < g.PD for i1, i2 in perm), name
        assert after < before and after <= warps + warps // 2, (name, before, after)
    # a perfect order exists for the zyx y- and x-sweeps (11 and 8 columns per bank)
    res = {t[0]: t for t in g.tables()}
    assert res["kLaneZyxS2"][5] == 11 and res["kLaneZyxS3"][5] == 8


def test_bank_model():
    # natural order of the xyz x-sweep: consecutive rows 23 floats apart,
    # conflict-free; the y-sweep pairs planes 22*23 apart, two-way conflicts
    g = _gen()
    cols, bank = g.phase_columns(0, 0)
    assert g.warp_passes(cols, bank) == 16
    cols, bank = g.phase_columns(0, 1)
    assert g.warp_passes(cols, bank) == 22
