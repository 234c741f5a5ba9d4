"""Write lane_maps.h: thread-to-column permutations of the FP32 sweeps.

The FP32 kernel keeps the padded 22^3 block of a patch group in shared
memory as [var][z][y][x] with row pitch XP = 23 floats and plane pitch
PP = 22 * 23 floats.  In a sweep every thread streams one 1-D column, and at
each step the 32 threads of a warp touch one cell of their 32 columns; two
threads whose cells fall in the same 4-byte bank (address mod 32) make the
access replay.  Taking the columns in their natural order (first transverse
index fastest) gives two-way conflicts in most sweeps.  This script orders
each sweep's columns so that consecutive groups of 32 (one warp) fall in
different banks where the column set allows it: columns are bucketed by
bank and every warp takes one column from each bank, fullest buckets first.

The x-sweep of an xyz set (already conflict-free in natural order) and the
z-sweep of an xyz set (whose threads write their finished columns to global
memory, where the natural order keeps the stores coalesced) are not
permuted.

Run: python gen_lane_maps.py  (rewrites lane_maps.h next to this file).
"""
import os

PD, NG, GS, XP = 22, 3, 16, 23
PP = PD * XP
STRIDE = (1, XP, PP)


def phase_columns(order: int, s: int):
    """Columns (i1, i2) of sweep s (0, 1, 2) of an xyz (0) or zyx (1) set in
    natural order, with the bank function of their cells."""
    ax = s if order == 0 else 2 - s
    t1 = 1 if ax == 0 else 0
    t2 = 1 if ax == 2 else 2
    done1 = (t1 < ax) if order == 0 else (t1 > ax)
    done2 = (t2 < ax) if order == 0 else (t2 > ax)
    lo1, n1 = (NG, GS) if done1 else (0, PD)
    lo2, n2 = (NG, GS) if done2 else (0, PD)
    cols = [(lo1 + c % n1, lo2 + c // n1) for c in range(n1 * n2)]

    def bank(col):
        return (col[0] * STRIDE[t1] + col[1] * STRIDE[t2]) % 32
    return cols, bank


def warp_passes(cols, bank):
    """Shared-memory passes of one access by every warp (max bank multiplicity)."""
    total = 0
    for w in range(0, len(cols), 32):
        cnt = [0] * 32
        for c in cols[w:w + 32]:
            cnt[bank(c)] += 1
        total += max(cnt)
    return total


def permute(cols, bank):
    buckets = {}
    for c in cols:
        buckets.setdefault(bank(c), []).append(c)
    out = []
    while len(out) < len(cols):
        warp = []
        for b in sorted(buckets, key=lambda b: (-len(buckets[b]), b)):
            if len(warp) == 32:
                break
            if buckets[b]:
                warp.append(buckets[b].pop(0))
        while len(warp) < 32 and any(buckets.values()):
            b = max(sorted(buckets), key=lambda b: len(buckets[b]))
            warp.append(buckets[b].pop(0))
        out += warp
    return out


# (name, order, sweep index) of the permuted sweeps
PHASES = (("kLaneXyzS2", 0, 1), ("kLaneZyxS1", 1, 0), ("kLaneZyxS2", 1, 1), ("kLaneZyxS3", 1, 2))


def tables():
    res = []
    for name, order, s in PHASES:
        cols, bank = phase_columns(order, s)
        perm = permute(cols, bank)
        res.append((name, order, s, perm, warp_passes(cols, bank), warp_passes(perm, bank), (len(cols) + 31) // 32))
    return res


def render() -> str:
    lines = ["// lane_maps.h -- written by gen_lane_maps.py; do not edit.",
             "// Thread-to-column order of the FP32 sweeps (see gen_lane_maps.py):",
             "// entry = i1 | i2 << 8, the column's two transverse padded indices.",
             "#pragma once", "", "namespace gh {", ""]
    for name, order, s, perm, before, after, warps in tables():
        lines.append(f"// {'xyz' if order == 0 else 'zyx'} sweep {s + 1}: {len(perm)} columns, "
                     f"shared-memory passes per access over its {warps} warps: {before} in natural order, {after} here")
        lines.append(f"__device__ const unsigned short {name}[{len(perm)}] = {{")
        vals = [str(i1 | (i2 << 8)) for i1, i2 in perm]
        for k in range(0, len(vals), 16):
            lines.append("    " + ", ".join(vals[k:k + 16]) + ",")
        lines.append("};")
        lines.append("")
    lines.append("}  // namespace gh")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lane_maps.h")
    with open(path, "w") as f:
        f.write(render())
    print(path)
