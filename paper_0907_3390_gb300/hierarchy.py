"""Patch-group hierarchies and neighbour maps (index bookkeeping only).

GAMER stores the mesh as an oct-tree of fixed 8^3-cell patches; the eight
children of a refined patch are allocated together, and each patch records
its parent, children and 26 siblings (Sec. 2.1).  The hydro solver works on
*patch groups*: the 2x2x2 octs of sibling patches, 16^3 interior cells
(Sec. 3.1).  This module builds, on the host, the static snapshot of such a
hierarchy that crosses the C ABI:

* per level, patch group ``g`` owns patches ``8g .. 8g+7``; the local patch
  index is ``(pz*2 + py)*2 + px``;
* ``nbr[g, d]`` for the 26 directions ``d = (dz+1)*9 + (dy+1)*3 + (dx+1)``
  (13, the group itself, skipped): a same-level patch-group index, ``-1`` if
  that region only exists on the coarser level (ghosts interpolated), or
  ``-2`` for an outflow (zero-gradient) domain face;
* ``parent[g]``: the patch on the level below whose children form group g;
* ``child[p]``: the patch group on the level above formed by the children of
  patch p, or -1.

Periodic wrap is encoded in the map itself.  Refinement obeys the
proper-nesting rule of Sec. 2.1: a patch is refined only if all 26 of its
same-level neighbours exist, so ghost cells never come from two levels down.

It also converts between whole-domain arrays ``[5][nz][ny][nx]`` and the
patch layout ``[5][8*n_groups][8][8][8]`` (x fastest).  Nothing here touches
the numerical method.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

NVAR = 5
PATCH = 8
GROUP = 16

DIRS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
        if (dx, dy, dz) != (0, 0, 0)]


def dir_index(dx: int, dy: int, dz: int) -> int:
    d = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
    return d if d < 13 else d - 1


@dataclass
class LevelMap:
    """Maps of one level.  ``coords[g]`` is the patch-group position in
    patch-group units of this level; ``dh`` the cell width."""
    n_groups: int
    dh: float
    nbr: np.ndarray                      # int32 [n_groups, 26]
    parent: np.ndarray | None            # int32 [n_groups] (None on level 0)
    child: np.ndarray | None = None      # int32 [8*n_groups] (None if finest)
    coords: np.ndarray = field(default=None)  # int64 [n_groups, 3]
    extent: tuple = (1, 1, 1)            # domain size in patch groups


def uniform_level(npg: tuple[int, int, int], dh: float = 1.0,
                  bc: tuple[str, str, str] = ("periodic",) * 3) -> LevelMap:
    """One level tiling an (npg_x, npg_y, npg_z) block of patch groups.
    Group index g = (gz*ny + gy)*nx + gx.  ``bc`` per axis: 'periodic' or
    'outflow'."""
    nx, ny, nz = npg
    n = nx * ny * nz
    coords = np.array([(g % nx, (g // nx) % ny, g // (nx * ny)) for g in range(n)],
                      dtype=np.int64).reshape(n, 3)
    nbr = np.empty((n, 26), dtype=np.int32)
    ext = (nx, ny, nz)
    for g in range(n):
        c = coords[g]
        for (dx, dy, dz) in DIRS:
            q = [c[0] + dx, c[1] + dy, c[2] + dz]
            val = None
            for a in range(3):
                if q[a] < 0 or q[a] >= ext[a]:
                    if bc[a] == "periodic":
                        q[a] %= ext[a]
                    else:
                        val = -2
            if val is None:
                val = (q[2] * ny + q[1]) * nx + q[0]
            nbr[g, dir_index(dx, dy, dz)] = val
    return LevelMap(n_groups=n, dh=dh, nbr=nbr, parent=None, coords=coords, extent=ext)


def domain_to_patches(arr: np.ndarray, npg: tuple[int, int, int]) -> np.ndarray:
    """[5][nz][ny][nx] whole-domain array -> [5][8*n_groups][8][8][8]."""
    nx, ny, nz = npg
    v = arr.shape[0]
    a = arr.reshape(v, nz, 2, PATCH, ny, 2, PATCH, nx, 2, PATCH)
    # axes: v, gz, pz, k, gy, py, j, gx, px, i  ->  v, gz, gy, gx, pz, py, px, k, j, i
    a = a.transpose(0, 1, 4, 7, 2, 5, 8, 3, 6, 9)
    return np.ascontiguousarray(a).reshape(v, 8 * nx * ny * nz, PATCH, PATCH, PATCH)


def patches_to_domain(p: np.ndarray, npg: tuple[int, int, int]) -> np.ndarray:
    """Inverse of :func:`domain_to_patches`."""
    nx, ny, nz = npg
    v = p.shape[0]
    a = p.reshape(v, nz, ny, nx, 2, 2, 2, PATCH, PATCH, PATCH)
    a = a.transpose(0, 1, 4, 7, 2, 5, 8, 3, 6, 9)
    return np.ascontiguousarray(a).reshape(v, nz * GROUP, ny * GROUP, nx * GROUP)


# ----------------------------------------------------------- hierarchies

@dataclass
class Hierarchy:
    levels: list[LevelMap]
    base_npg: tuple[int, int, int]
    L: float = 1.0   # domain side length (cubic cells)

    @property
    def n_levels(self) -> int:
        return len(self.levels)

    def patch_counts(self) -> list[int]:
        return [8 * lv.n_groups for lv in self.levels]

    def cell_centres(self, level: int) -> np.ndarray:
        """[3][8*n_groups][8][8][8] cell-centre coordinates of a level."""
        lv = self.levels[level]
        dh = lv.dh
        lp = np.arange(8)
        pofs = np.stack([lp & 1, (lp >> 1) & 1, (lp >> 2) & 1], axis=1)      # [8, 3]
        corner = ((lv.coords[:, None, :] * 2 + pofs[None]) * PATCH * dh).reshape(-1, 3)
        off = (np.arange(PATCH) + 0.5) * dh
        x = corner[:, 0, None, None, None] + off[None, None, None, :]
        y = corner[:, 1, None, None, None] + off[None, None, :, None]
        z = corner[:, 2, None, None, None] + off[None, :, None, None]
        return np.stack(np.broadcast_arrays(x, y, z))


def _patch_key(level_coords, lp):
    px, py, pz = lp & 1, (lp >> 1) & 1, (lp >> 2) & 1
    return (2 * level_coords[0] + px, 2 * level_coords[1] + py, 2 * level_coords[2] + pz)


def patch_neighbours(level: LevelMap) -> np.ndarray:
    """int64 [8 n_groups, 27]: for patch p and offset bit
    b = (dz+1)*9 + (dy+1)*3 + (dx+1), the patch of the same level at offset
    (dx, dy, dz) from p, found through the group map; column 13 is p itself,
    -1 marks a region that exists only on the coarser level and -2 one
    outside the domain (an outflow face)."""
    n = level.n_groups
    lp = np.arange(8)
    loc = np.stack([lp & 1, (lp >> 1) & 1, lp >> 2], axis=1)                       # [8, 3]
    offs = np.array([[b % 3 - 1, (b // 3) % 3 - 1, b // 9 - 1] for b in range(27)])  # [27, 3]
    s = loc[:, None, :] + offs[None, :, :]                                          # [8, 27, 3]
    go = np.where(s < 0, -1, np.where(s > 1, 1, 0))                                 # group offset
    q = s - 2 * go                                                                  # patch in that group
    lq = (q[..., 2] * 2 + q[..., 1]) * 2 + q[..., 0]                                # [8, 27]
    gb = (go[..., 2] + 1) * 9 + (go[..., 1] + 1) * 3 + (go[..., 0] + 1)             # [8, 27]
    nbr = np.asarray(level.nbr, dtype=np.int64).reshape(n, 26)
    gt = np.concatenate([nbr[:, :13], np.arange(n, dtype=np.int64)[:, None], nbr[:, 13:]], axis=1)
    h = gt[:, gb]                                                                   # [n, 8, 27]
    return np.where(h >= 0, 8 * h + lq[None], h).reshape(8 * n, 27)


def build_hierarchy(base_npg: tuple[int, int, int], score_fn, n_levels: int,
                    targets=None, L: float = 1.0,
                    bc: tuple[str, str, str] = ("periodic",) * 3) -> Hierarchy:
    """Build a properly nested hierarchy over a base level with the given
    boundaries.

    ``score_fn(level, centres)`` receives the cell centres [3][8n][8][8][8]
    of a level and returns a refinement score per patch (shape [8n]); a
    patch with a positive score asks for refinement.  A patch is eligible
    only if its 26 same-level neighbours all exist (proper nesting; a region
    outside the domain at an outflow face counts as present).  When
    ``targets`` is given, level l+1 is made of the children of the
    ``targets[l+1] // 8`` eligible patches with the highest scores.  Patch
    groups of the new level are numbered in the order of their parents."""
    nx, ny, nz = base_npg
    lv0 = uniform_level(base_npg, dh=L / (GROUP * nx), bc=bc)
    levels = [lv0]
    H = Hierarchy(levels=levels, base_npg=base_npg, L=L)
    for lev in range(n_levels - 1):
        cur = levels[-1]
        score = np.asarray(score_fn(lev, H.cell_centres(lev)), dtype=np.float64)
        eligible = np.nonzero(np.all(patch_neighbours(cur) != -1, axis=1))[0]
        if targets is not None:
            want = int(targets[lev + 1]) // 8
            order = np.argsort(-score[eligible], kind="stable")
            refine = np.sort(eligible[order[:want]]).tolist()
        else:
            refine = [int(p) for p in eligible if score[p] > 0]
        if not refine:
            break
        levels.append(refine_level(cur, refine))
    return H


def refine_level(cur: LevelMap, refine) -> LevelMap:
    """The next finer level made of the children of the listed patches of
    ``cur`` (one patch group per refined patch, numbered in list order);
    sets ``cur.child``.  The new group's neighbour in direction d is the
    child group of the patch next to its parent in direction d (-1 if that
    patch is not refined, -2 outside the domain).  Every refined patch must
    have its 26 same-level neighbours."""
    refine = np.asarray([int(p) for p in refine], dtype=np.int64)
    child = np.full(8 * cur.n_groups, -1, dtype=np.int32)
    child[refine] = np.arange(len(refine), dtype=np.int32)
    cur.child = child
    pn = patch_neighbours(cur)[refine]
    pn = np.concatenate([pn[:, :13], pn[:, 14:]], axis=1)                           # [n_f, 26]
    if np.any(pn == -1):
        raise ValueError("refined patch without its 26 same-level neighbours")
    nbr = np.where(pn >= 0, child[np.maximum(pn, 0)], pn).astype(np.int32)
    g, lp = refine // 8, refine % 8
    loc = np.stack([lp & 1, (lp >> 1) & 1, lp >> 2], axis=1)
    fine_coords = (2 * np.asarray(cur.coords, dtype=np.int64)[g] + loc).reshape(len(refine), 3)
    ext_p = tuple(2 * e for e in cur.extent)
    return LevelMap(n_groups=len(refine), dh=cur.dh / 2, nbr=nbr, parent=refine.astype(np.int32),
                    coords=fine_coords, extent=ext_p)


def patch_lookup(level: LevelMap) -> dict:
    """{(px, py, pz) patch coordinates on the level: patch index}."""
    out = {}
    for g in range(level.n_groups):
        for lp in range(8):
            out[_patch_key(level.coords[g], lp)] = 8 * g + lp
    return out


def leaf_mask(level: LevelMap) -> np.ndarray:
    """bool [8*n_groups]: patches without children."""
    if level.child is None:
        return np.ones(8 * level.n_groups, dtype=bool)
    return level.child < 0


def validate_level(levels: list[LevelMap], l: int) -> None:
    """Host-side consistency check of one level's maps (raises ValueError)."""
    lv = levels[l]
    n = lv.n_groups
    if lv.nbr.shape != (n, 26):
        raise ValueError("nbr shape")
    if np.any(lv.nbr >= n) or np.any(lv.nbr < -2):
        raise ValueError("nbr out of range")
    if l == 0 and np.any(lv.nbr == -1):
        raise ValueError("coarse neighbour on the base level")
    if l > 0:
        if lv.parent is None or lv.parent.shape != (n,):
            raise ValueError("parent")
        if np.any(lv.parent < 0) or np.any(lv.parent >= 8 * levels[l - 1].n_groups):
            raise ValueError("parent out of range")
