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
              neighbours all exist (proper nesting; a neighbour region
              outside the domain at an outflow face counts as present;
              patches that fail are unflagged); a new patch group inherits
              the data of the old group with the same position where there
              was one, and is otherwise filled by Min-Mod interpolation
              from its parent level (orc_refine_fill).

The maps of every rebuilt level (group coordinates, parents, the children
of the level below, the 26-neighbour map) are built here from the maps of
the level below by walking patch by patch through its neighbour map, with
no code shared with the library's own bookkeeping.  Only the hierarchy
given as input comes from the input generators.

The levels above ``max_levels`` - 1 are never created.
"""
from __future__ import annotations

import copy
from dataclasses import dataclass

import numpy as np

from . import OracleLevels

# offset of mask bit b = (dz+1)*9 + (dy+1)*3 + (dx+1); bit 13 is the patch itself
_OFFS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _dir(dx: int, dy: int, dz: int) -> int:
    """Column of a direction in a 26-neighbour map (13, the group itself, skipped)."""
    d = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
    return d if d < 13 else d - 1


@dataclass
class Level:
    """One level of a rebuilt hierarchy: the fields the oracle and the tests
    read (the same names as the input hierarchy's levels)."""
    n_groups: int
    dh: float
    nbr: np.ndarray            # int32 [n_groups, 26]
    parent: np.ndarray | None  # int32 [n_groups], None on level 0
    child: np.ndarray | None   # int32 [8 n_groups], None if no finer level
    coords: np.ndarray         # int64 [n_groups, 3], in patch groups of this level
    extent: tuple              # domain size in patch groups of this level


@dataclass
class Hierarchy:
    levels: list
    base_npg: tuple
    L: float = 1.0

    @property
    def n_levels(self) -> int:
        return len(self.levels)


def _own_level(lv) -> Level:
    """A private copy of an input level."""
    return Level(n_groups=int(lv.n_groups), dh=float(lv.dh), nbr=np.array(lv.nbr, dtype=np.int32),
                 parent=None if lv.parent is None else np.array(lv.parent, dtype=np.int32),
                 child=None if lv.child is None else np.array(lv.child, dtype=np.int32),
                 coords=np.array(lv.coords, dtype=np.int64).reshape(-1, 3), extent=tuple(lv.extent))


def patch_neighbour(level, p: int, dx: int, dy: int, dz: int) -> int:
    """The patch at offset (dx, dy, dz) from patch p of the same level,
    found through the level's group map: a patch index, -1 where that region
    exists only on the coarser level, -2 outside the domain (outflow face).
    Patch p = 8 g + (pz*2 + py)*2 + px sits at (px, py, pz) in group g."""
    g, lp = divmod(int(p), 8)
    loc = (lp & 1, (lp >> 1) & 1, (lp >> 2) & 1)
    go, q = [], []
    for a, d in enumerate((dx, dy, dz)):
        s = loc[a] + d                       # -1 .. 2 in units of patches
        o = -1 if s < 0 else (1 if s > 1 else 0)
        go.append(o)
        q.append(s - 2 * o)
    if go == [0, 0, 0]:
        h = g
    else:
        h = int(level.nbr[g][_dir(*go)])
        if h < 0:
            return h
    return 8 * h + (q[2] * 2 + q[1]) * 2 + q[0]


def patch_coords(level) -> dict:
    """patch index -> (px, py, pz), its position in patches of its level."""
    out = {}
    for g in range(level.n_groups):
        c = [int(v) for v in level.coords[g]]
        for lp in range(8):
            out[8 * g + lp] = (2 * c[0] + (lp & 1), 2 * c[1] + ((lp >> 1) & 1), 2 * c[2] + ((lp >> 2) & 1))
    return out


_patch_coords = patch_coords


def combine_masks(level, masks) -> set:
    """Positions of the patches of a level that a flag reaches: patch p's
    mask bit b points at the patch at offset _OFFS[b] from p (flags that
    point outside the domain or at a region not on this level are dropped)."""
    pc = patch_coords(level)
    flagged = set()
    for p, m in enumerate(masks):
        m = int(m)
        if m == 0:
            continue
        for b, (dx, dy, dz) in enumerate(_OFFS):
            if (m >> b) & 1:
                q = patch_neighbour(level, p, dx, dy, dz)
                if q >= 0:
                    flagged.add(pc[q])
    return flagged


def properly_nested(level, p: int) -> bool:
    """Whether all 26 same-level neighbours of patch p exist (or lie outside
    the domain at an outflow face), so that the ghost cells of its children
    never come from two levels down (Sec. 2.1)."""
    return all(patch_neighbour(level, p, dx, dy, dz) != -1 for (dx, dy, dz) in _OFFS if (dx, dy, dz) != (0, 0, 0))


def refine_maps(cur: Level, refine) -> tuple[Level, np.ndarray]:
    """The level made of the children of the listed patches of cur: the
    eight children of a patch are allocated together (Sec. 2.1), so refined
    patch refine[i] becomes patch group i of the new level.  Returns the new
    level (coordinates, parents, 26-neighbour map: the children of the
    corresponding neighbour patch of cur, -1 where that patch is not
    refined, -2 outside the domain) and the child map of cur."""
    refine = [int(p) for p in refine]
    child = np.full(8 * cur.n_groups, -1, dtype=np.int32)
    for i, p in enumerate(refine):
        child[p] = i
    pc = patch_coords(cur)
    nbr = np.empty((len(refine), 26), dtype=np.int32)
    for i, p in enumerate(refine):
        for (dx, dy, dz) in _OFFS:
            if (dx, dy, dz) == (0, 0, 0):
                continue
            q = patch_neighbour(cur, p, dx, dy, dz)
            if q == -1:
                raise ValueError(f"patch {p} is not properly nested")
            nbr[i, _dir(dx, dy, dz)] = -2 if q == -2 else int(child[q])
    coords = np.array([pc[p] for p in refine], dtype=np.int64).reshape(len(refine), 3)
    fine = Level(n_groups=len(refine), dh=cur.dh / 2, nbr=nbr, parent=np.array(refine, dtype=np.int32),
                 child=None, coords=coords, extent=tuple(2 * e for e in cur.extent))
    return fine, child


def regrid(H, states, gamma: float, criterion: int, thresholds, n_buffer: int, max_levels: int):
    """New (hierarchy, states) after one rebuild of the refinement map; the
    flags are decided in double precision (orc_flag_level)."""
    O = OracleLevels(H, states)
    n_old = H.n_levels
    n_flag = min(n_old, max_levels - 1)
    flags = [combine_masks(H.levels[l], O.flag_level(l, gamma, criterion, thresholds[l], n_buffer))
             for l in range(n_flag)]
    # a patch with a flagged child stays flagged (finest to coarsest)
    for l in range(n_flag - 2, -1, -1):
        for k in flags[l + 1]:
            flags[l].add((k[0] // 2, k[1] // 2, k[2] // 2))
    base = _own_level(H.levels[0])
    base.child = None
    levels = [base]
    new_states = [np.array(states[0], dtype=np.float64, copy=True)]
    for l in range(n_flag):
        cur = levels[l]
        pc = patch_coords(cur)
        refine = [p for p in range(8 * cur.n_groups) if pc[p] in flags[l] and properly_nested(cur, p)]
        if not refine:
            break
        fine, cur.child = refine_maps(cur, refine)
        # inherit the old fine group with the same coordinates, if any
        inherit = np.full(fine.n_groups, -1, dtype=np.int32)
        if l + 1 < n_old:
            old = H.levels[l + 1]
            pos = {tuple(int(c) for c in old.coords[g]): g for g in range(old.n_groups)}
            for i in range(fine.n_groups):
                inherit[i] = pos.get(tuple(int(c) for c in fine.coords[i]), -1)
        On = OracleLevels(Hierarchy(levels=levels, base_npg=H.base_npg, L=H.L), new_states, with_flux=False)
        new_states.append(On.refine_fill(l, fine.parent, inherit, states[l + 1] if l + 1 < n_old else None))
        levels.append(fine)
    return Hierarchy(levels=levels, base_npg=H.base_npg, L=H.L), new_states
