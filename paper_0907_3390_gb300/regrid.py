"""Rebuild of the refinement map (Sec. 2.1 step 4) through the C ABI.

The two sweeps over the data run on the device: the flag step
(``gamer_hydro_flag``: per-cell criterion and flag buffer, reduced to one
mask per patch) and the data of every rebuilt level
(``gamer_hydro_refine_fill``: inherited groups copied, new ones filled by
Min-Mod interpolation).  What lies between is bookkeeping on the host, as
GAMER does it on the CPU (readings R21-R23):

* a patch is flagged when its own mask or the mask of one of its 26
  siblings has the bit pointing at it;
* from the finest level down, a patch with a flagged child stays flagged;
* from level 0 up, the new level l+1 is made of the children of the flagged
  patches of the new level l whose 26 same-level neighbours exist (proper
  nesting); a new group inherits the old group with the same position.
"""
from __future__ import annotations

import numpy as np

from . import binding as B
from . import hierarchy as hm

def patch_coords(level) -> np.ndarray:
    """[8 n_groups, 3] patch coordinates of a level (patch index order)."""
    lp = np.arange(8)
    local = np.stack([lp & 1, (lp >> 1) & 1, lp >> 2], axis=1)
    return (2 * np.asarray(level.coords, dtype=np.int64)[:, None, :] + local[None]).reshape(-1, 3)


def _keys(c, ext):
    return (c[:, 2] * ext[1] + c[:, 1]) * ext[0] + c[:, 0]


def flagged_patches(level, masks: np.ndarray) -> np.ndarray:
    """bool [8 n_groups]: patches reached by a mask bit of their own or of a
    sibling (mask bit b of patch p points at the patch at offset b of p;
    bits that point outside the domain or off the level are dropped)."""
    pn = hm.patch_neighbours(level)
    out = np.zeros(pn.shape[0], dtype=bool)
    m = masks.astype(np.uint64)
    for b in range(27):
        src = np.nonzero((m >> np.uint64(b)) & np.uint64(1))[0]
        tgt = pn[src, b]
        out[tgt[tgt >= 0]] = True
    return out


def _nested(level) -> np.ndarray:
    """bool [8 n_groups]: patches whose 26 same-level neighbours all exist
    (a region outside the domain at an outflow face counts as present)."""
    return np.all(hm.patch_neighbours(level) != -1, axis=1)


def rebuild(S, D, criterion: int, thresholds, n_buffer: int, max_levels: int):
    """New DeviceHierarchy after one rebuild of the refinement map of D
    (handle S, whose precision is D's); D itself is left as it was."""
    import torch
    H = D.H
    dev = D.u[0].device
    n_old = H.n_levels
    n_flag = min(n_old, max_levels - 1)
    flag_sets = []
    for l in range(n_flag):
        masks = torch.empty(8 * H.levels[l].n_groups, dtype=torch.int32, device=dev)
        B.gamer_hydro_flag(S.h, D, l, criterion, float(thresholds[l]), n_buffer, masks)
        m = masks.cpu().numpy().view(np.uint32)
        pc = patch_coords(H.levels[l])
        flag_sets.append({tuple(int(v) for v in c) for c in pc[flagged_patches(H.levels[l], m)]})
    for l in range(n_flag - 2, -1, -1):
        flag_sets[l] |= {(k[0] // 2, k[1] // 2, k[2] // 2) for k in flag_sets[l + 1]}
    import copy
    base = copy.deepcopy(H.levels[0])
    base.child = None
    levels = [base]
    states = [D.u[0].clone()]
    plans = []
    for l in range(n_flag):
        cur = levels[l]
        pc = patch_coords(cur)
        want = np.array([tuple(int(v) for v in c) in flag_sets[l] for c in pc], dtype=bool)
        refine = np.nonzero(want & _nested(cur))[0]
        if len(refine) == 0:
            break
        fine = hm.refine_level(cur, refine)
        inherit = np.full(fine.n_groups, -1, dtype=np.int32)
        if l + 1 < n_old:
            old = H.levels[l + 1]
            ext = np.array(old.extent, dtype=np.int64)
            ko = _keys(np.asarray(old.coords, dtype=np.int64), ext)
            kn = _keys(np.asarray(fine.coords, dtype=np.int64), ext)
            order = np.argsort(ko)
            pos = np.minimum(np.searchsorted(ko[order], kn), len(ko) - 1)
            hit = ko[order][pos] == kn
            inherit[hit] = order[pos[hit]]
        levels.append(fine)
        plans.append((fine, inherit))
    Hn = hm.Hierarchy(levels=levels, base_npg=H.base_npg, L=H.L)
    for l, (fine, inherit) in enumerate(plans):
        states.append(torch.empty((5, 8 * fine.n_groups, 8, 8, 8), dtype=D.dtype, device=dev))
    Dn = B.DeviceHierarchy(Hn, states, D.dtype, device=dev)
    for l, (fine, inherit) in enumerate(plans):
        pn = torch.as_tensor(np.asarray(fine.parent, dtype=np.int32), device=dev)
        ih = torch.as_tensor(inherit, device=dev)
        u_old = D.u[l + 1] if l + 1 < n_old else None
        B.gamer_hydro_refine_fill(S.h, Dn, l, pn, ih, u_old, Dn.u[l + 1])
    torch.cuda.synchronize()
    return Dn
