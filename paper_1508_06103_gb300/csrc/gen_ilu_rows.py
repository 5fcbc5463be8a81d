"""Generate ilu_rows.inc: straight-line ILU(0) elimination of one KKT row per thread.

Every row of the space-time KKT matrix is one of three types (C, G, f) with
a fixed structural stencil of slots (level offset dt, spatial offset, column
component), ordered as the columns are ordered.  The IKJ elimination of a row
is therefore the same fixed sequence of operations for every row of a type:

    for each L-slot s in order:      a_s <- a_s / u_kk(s)
        for each U-slot t of the pivot row k(s) whose column is in the row:
                                     a_s2 <- a_s2 - a_s * u_k[t]

This script writes that sequence out as device code with compile-time slot
indices, so one thread eliminates one row with the row in registers and the
pivot-row entries read straight from memory.  The code has no branches: a
pivot point outside the subdomain box is pointed at a stored unit row (1 on
the diagonals, 0 elsewhere), so its column (which holds 0) contributes
nothing, and all loads can be issued early.

The slot order here must equal the one the library builds at run time
(ras.cu, build_tables); the generated header carries the per-type counts and
a checksum of the slot list that the library verifies.

    python gen_ilu_rows.py      # rewrites ilu_rows.inc next to this file
"""

from __future__ import annotations

import os

HERE = os.path.dirname(os.path.abspath(__file__))


def slot_tables():
    slots, base, diag, count = [], {}, {}, {}
    for c in range(3):
        base[c] = len(slots)
        dt_lo = 0 if c == 1 else -1
        dt_hi = 0 if c == 0 else 1
        for dt in range(dt_lo, dt_hi + 1):
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        for cc in range(3):
                            if c == 0:
                                use = cc in (0, 2)
                            elif c == 1:
                                use = cc == 1 or (cc == 0 and dx == dy == dz == 0)
                            else:
                                use = cc in (1, 2)
                            if not use:
                                continue
                            if dt == dz == dy == dx == 0 and cc == c:
                                diag[c] = len(slots)
                            slots.append((dt, dz, dy, dx, cc))
        count[c] = len(slots) - base[c]
    return slots, base, diag, count


def checksum(slots):
    h = 0
    for i, (dt, dz, dy, dx, cc) in enumerate(slots):
        h = (h * 131 + (i + 1) * (dt + 2) * 7 + (dz + 2) * 11 + (dy + 2) * 13 + (dx + 2) * 17 + cc * 19) % 1000000007
    return h


def generate() -> str:
    slots, base, diag, count = slot_tables()
    index = {}
    for c in range(3):
        for s in range(base[c], base[c] + count[c]):
            index[(c,) + slots[s]] = s
    out = [
        "// Generated by gen_ilu_rows.py from the KKT row stencils -- do not edit by hand.",
        "// Straight-line IKJ ILU(0) elimination of one row of each type (C, G, f).",
        "#pragma once",
        "",
        f"constexpr long long kGenSlotChecksum = {checksum(slots)}LL;",
        "",
    ]
    nbr_tables = []
    for c in range(3):
        # distinct pivot points (offsets) of the L-slots, in first-use order
        nbrs = []
        for s in range(base[c], diag[c]):
            off = slots[s][:4]
            if off not in nbrs:
                nbrs.append(off)
        nbr_tables.append(nbrs)
        nupd = 0
        body = []
        for s in range(base[c], diag[c]):
            dt, dz, dy, dx, ck = slots[s]
            i = nbrs.index((dt, dz, dy, dx))
            ls = s - base[c]
            ups = []
            for t in range(diag[ck] + 1, base[ck] + count[ck]):
                key = (c, dt + slots[t][0], dz + slots[t][1], dy + slots[t][2], dx + slots[t][3], slots[t][4])
                if key in index:
                    ups.append((t, index[key] - base[c]))
            nupd += len(ups)
            body.append(f"  {{  // slot {s}: pivot row {'CGf'[ck]} at offset {(dt, dz, dy, dx)}")
            body.append(f"    const T* u = F + nb[{i} * NS];")
            body.append(f"    const int st = ns[{i} * NS];")
            body.append(f"    const T l = a[{ls}] / u[{diag[ck]} * st];")
            body.append(f"    a[{ls}] = l;")
            for t, s2 in ups:
                body.append(f"    a[{s2}] -= l * u[{t} * st];")
            body.append("  }")
        out.append(f"// row type {'CGf'[c]}: {count[c]} slots, {diag[c] - base[c]} L-slots, {nupd} updates, "
                   f"{len(nbrs)} pivot points")
        out.append(f"constexpr int kGenRowSlots{c} = {count[c]};")
        out.append(f"constexpr int kGenRowNbrs{c} = {len(nbrs)};")
        out.append(f"constexpr int kGenRowUpdates{c} = {nupd};")
        out.append("// nb[i * NS]: offset of pivot point i's column in F (the unit row outside the box),")
        out.append("// ns[i * NS]: row stride of its level block")
        out.append("template <typename T, int NS>")
        out.append(f"__device__ __forceinline__ void ilu_elim_row{c}(T* a, const T* __restrict__ F, "
                   "const int* nb, const int* ns) {")
        out.extend(body)
        out.append("}")
        out.append("")
    # neighbour offset tables (dt, dz, dy, dx) per row type
    mx = max(len(n) for n in nbr_tables)
    out.append(f"constexpr int kGenMaxNbrs = {mx};")
    out.append("__constant__ signed char c_gen_nbr[3][%d][4] = {" % mx)
    for c in range(3):
        rows = [f"{{{dt}, {dz}, {dy}, {dx}}}" for (dt, dz, dy, dx) in nbr_tables[c]]
        rows += ["{0, 0, 0, 0}"] * (mx - len(rows))
        out.append("    {" + ", ".join(rows) + "},")
    out.append("};")
    return "\n".join(out) + "\n"


if __name__ == "__main__":
    path = os.path.join(HERE, "ilu_rows.inc")
    with open(path, "w") as fh:
        fh.write(generate())
    print(path)
