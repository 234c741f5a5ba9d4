"""Host bookkeeping of the refinement-map rebuild (Sec. 2.1 step 4) in the
library's Python layer against the oracle's own construction, on the CPU:
the rebuilt level's coordinates, parents, child map and 26-neighbour map,
which patches a set of flag masks reaches, and which patches are properly
nested, on periodic and outflow domains over two successive levels."""
import numpy as np
import pytest

from oracle import regrid as org
from paper_0907_3390_gb300 import hierarchy as hm
from paper_0907_3390_gb300 import regrid as rg
from paper_0907_3390_gb300 import workloads as wl


@pytest.mark.parametrize("bc", [("periodic",) * 3, ("outflow", "periodic", "outflow"), ("outflow",) * 3])
def test_rebuilt_maps_match_oracle(bc):
    rng = np.random.default_rng(11)
    H = wl.uniform_hierarchy((3, 2, 2), bc=bc)
    mine = H.levels[0]
    ref = org._own_level(H.levels[0])
    for lev in range(2):
        nested = np.nonzero(rg._nested(mine))[0]
        want = [p for p in range(8 * ref.n_groups) if org.properly_nested(ref, p)]
        assert nested.tolist() == want
        refine = sorted(rng.choice(want, size=max(1, (2 * len(want)) // 3), replace=False).tolist())
        fine = hm.refine_level(mine, refine)
        fref, child = org.refine_maps(ref, refine)
        assert np.array_equal(mine.child, child)
        assert np.array_equal(fine.nbr, fref.nbr)
        assert np.array_equal(fine.parent, fref.parent)
        assert np.array_equal(np.asarray(fine.coords), fref.coords)
        assert fine.extent == fref.extent and fine.dh == fref.dh
        # flag masks: random bits on random patches
        masks = np.zeros(8 * fine.n_groups, dtype=np.uint32)
        pick = rng.choice(len(masks), size=len(masks) // 3, replace=False)
        masks[pick] = rng.integers(0, 1 << 27, size=len(pick), dtype=np.uint64).astype(np.uint32)
        got = rg.flagged_patches(fine, masks)
        pc = org.patch_coords(fref)
        reached = org.combine_masks(fref, masks)
        assert {pc[p] for p in np.nonzero(got)[0]} == reached
        mine, ref = fine, fref
