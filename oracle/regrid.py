"""Rebuild of the refinement map (Sec. 2.1 step 4), oracle side.

Test infrastructure: used only by the tests.  Follows the paper's two
sub-steps with readings R21-R23:

flag step     every patch of level l gets the flags of orc_flag_level: a
              patch is flagged when a cell of its own, or the flag buffer
              of a cell of one of its 26 siblings, reaches it; then, from
              the finest level down, a patch with a flagged child stays
              flagged (the fine data are preserved);
refinement    from level 0 up, the new level l+1 is made of the children of
step          the flagged patches of the new level l whose 26 same-level
              neighbours all exist (proper nesting; patches that fail are
              unflagged); a new patch group inherits the data of the old
              group with the same parent where there was one, and is
              otherwise filled by Min-Mod interpolation from its parent
              level (orc_refine_fill).

The levels above ``max_levels`` - 1 are never created.
"""
from __future__ import annotations

import numpy as np

from . import OracleLevels
from paper_0907_3390_gb300 import hierarchy as hm

_OFFS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _patch_coords(level):
    """patch index -> (px, py, pz) on its level."""
    out = {}
    for g in range(level.n_groups):
        for lp in range(8):
            out[8 * g + lp] = (2 * int(level.coords[g][0]) + (lp & 1), 2 * int(level.coords[g][1]) + ((lp >> 1) & 1),
                               2 * int(level.coords[g][2]) + ((lp >> 2) & 1))
    return out


def combine_masks(level, masks) -> set:
    """Coordinates of the flagged patches of a level from its masks."""
    coords = _patch_coords(level)
    ext = [2 * e for e in level.extent]
    flagged = set()
    for p, m in enumerate(masks):
        if m == 0:
            continue
        k = coords[p]
        for bit, (dx, dy, dz) in enumerate(_OFFS):
            if (int(m) >> bit) & 1:
                flagged.add(((k[0] + dx) % ext[0], (k[1] + dy) % ext[1], (k[2] + dz) % ext[2]))
    present = set(coords.values())
    return flagged & present


def regrid(H, states, gamma: float, criterion: int, thresholds, n_buffer: int, max_levels: int,
           single: bool = False):
    """New (hierarchy, states) after one rebuild of the refinement map;
    single: flags of a single-precision run (criteria in float)."""
    O = OracleLevels(H, states)
    n_old = H.n_levels
    n_flag = min(n_old, max_levels - 1)
    flags = [combine_masks(H.levels[l], O.flag_level(l, gamma, criterion, thresholds[l], n_buffer, single))
             for l in range(n_flag)]
    # a patch with a flagged child stays flagged (finest to coarsest)
    for l in range(n_flag - 2, -1, -1):
        for k in flags[l + 1]:
            flags[l].add((k[0] // 2, k[1] // 2, k[2] // 2))
    # rebuild from level 0 up
    import copy
    base = copy.deepcopy(H.levels[0])
    base.child = None
    levels = [base]
    new_states = [np.array(states[0], dtype=np.float64, copy=True)]
    for l in range(n_flag):
        cur = levels[l]
        coords = _patch_coords(cur)
        lookup = {v: k for k, v in coords.items()}
        ext = [2 * e for e in cur.extent]
        refine = []
        for p in range(8 * cur.n_groups):
            k = coords[p]
            if k not in flags[l]:
                continue
            if all(((k[0] + dx) % ext[0], (k[1] + dy) % ext[1], (k[2] + dz) % ext[2]) in lookup
                   for (dx, dy, dz) in _OFFS if (dx, dy, dz) != (0, 0, 0)):
                refine.append(p)
        if not refine:
            break
        fine = hm.refine_level(cur, refine)
        # inherit the old fine group with the same coordinates, if any
        inherit = np.full(fine.n_groups, -1, dtype=np.int32)
        if l + 1 < n_old:
            old = H.levels[l + 1]
            pos = {tuple(int(c) for c in old.coords[g]): g for g in range(old.n_groups)}
            for i in range(fine.n_groups):
                inherit[i] = pos.get(tuple(int(c) for c in fine.coords[i]), -1)
        On = OracleLevels(hm.Hierarchy(levels=levels, base_npg=H.base_npg, L=H.L), new_states, with_flux=False)
        new_states.append(On.refine_fill(l, fine.parent, inherit, states[l + 1] if l + 1 < n_old else None))
        levels.append(fine)
    Hn = hm.Hierarchy(levels=levels, base_npg=H.base_npg, L=H.L)
    return Hn, new_states
