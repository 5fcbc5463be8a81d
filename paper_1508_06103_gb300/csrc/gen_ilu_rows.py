"""Generate ilu_rows.inc: straight-line ILU(0) elimination of one KKT row per thread.

(and ilu_slots.inc: the slot list's checksum and each slot's row in a chunk block,
also indexed by the slot's offsets for the value gather)

Every row of the space-time KKT matrix is one of three types (C, G, f) with
a fixed structural stencil of slots (level offset dt, spatial offset, column
component), ordered as the columns are ordered.  The IKJ elimination of a row
is therefore the same fixed sequence of operations for every row of a type:

    for each L-slot s in order:      a_s <- a_s / u_kk(s)
        for each U-slot t of the pivot row k(s) whose column is in the row:
                                     a_s2 <- a_s2 - a_s * u_k[t]

This script writes that elimination out as device code with compile-time slot
indices, one target entry at a time: entry x of the row receives its updates
a_x <- a_x - l_s * u_k(s)[t] in increasing L-slot order s (the order IKJ
applies them), and an L-entry is then scaled by its pivot's reciprocal.  The diagonal slot of a
finished row holds 1/u_kk rather than u_kk, so a row costs one division
instead of one per L-slot: a division expands to code with a branch, which
would stop loads from being issued ahead of it.  Only the multipliers l_s
stay live in registers; each entry is read, finished and stored in one go, which leaves
registers for many pivot-row loads in flight.  The code has no branches: a
pivot point outside the subdomain box is pointed at a stored unit row (1 on
the diagonals, 0 elsewhere), so its column (which holds 0) contributes
nothing, and all loads can be issued early.

The slot order here must equal the one the library builds at run time
(ras.cu, build_tables); the generated header carries the per-type counts and
a checksum of the slot list that the library verifies.

    python gen_ilu_rows.py      # rewrites ilu_slots.inc and ilu_rows.inc next to this file
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


def slot_rank(s, base, diag, count):
    """Row of slot s in a chunk block: the L-slots of C, G, f, then the diagonal
    and U-slots of C, G, f (the order the subdomain solve streams them in)."""
    nl = [diag[c] - base[c] for c in range(3)]
    nu = [count[c] - nl[c] for c in range(3)]
    for c in range(3):
        if base[c] <= s < diag[c]:
            return sum(nl[:c]) + (s - base[c])
    for c in range(3):
        if diag[c] <= s < base[c] + count[c]:
            return sum(nl) + sum(nu[:c]) + (s - diag[c])
    raise ValueError(s)


def checksum(slots):
    h = 0
    for i, (dt, dz, dy, dx, cc) in enumerate(slots):
        h = (h * 131 + (i + 1) * (dt + 2) * 7 + (dz + 2) * 11 + (dy + 2) * 13 + (dx + 2) * 17 + cc * 19) % 1000000007
    return h


GROUP32 = 8    # entries finished between two rounds of stores, FP32
GROUP64 = 4    # the same in FP64 (twice the registers per value)


def row_function(c, prec, group, nl, cnt, base, slots, diag, rank, nbrs, contrib):
    """Device code eliminating one row of type c.

    The compiler cannot move a global load above a global store, so the
    entries are finished in groups of `group`, each group's values stored
    after all of its loads: a window of loads can be in flight at a time, and
    the group bounds the registers they take.  The multipliers l_s stay in
    registers for the rest of the row.
    """
    o = [
        "// own: the point's column in its chunk block (row stride ost); F + nb[i * NS].x: pivot point i's",
        "// column (the unit row outside the box), nb[i * NS].y: its row stride.  Stores 1/pivot in the",
        "// diagonal slot and returns the pivot.",
        "template <typename T, int NS>",
        f"__device__ __forceinline__ T ilu_row{c}_{prec}(T* __restrict__ own, const int ost, "
        "const T* __restrict__ F, const int2* __restrict__ nb) {",
        f"  T l[{nl}], u[{group}], d;",
    ]

    def accumulate(x, dst):
        o.append("  {")
        o.append(f"    T acc = own[{rank[base + x]} * ost];")
        for (s, i, t) in contrib[x]:
            o.append(f"    {{ const int2 q = nb[{i} * NS]; acc -= l[{s}] * F[q.x + {rank[t]} * q.y]; }}")
        if x < nl:
            dt, dz, dy, dx, ck = slots[base + x]
            i = nbrs.index((dt, dz, dy, dx))
            o.append(f"    {{ const int2 q = nb[{i} * NS]; l[{x}] = acc * F[q.x + {rank[diag[ck]]} * q.y]; }}")
        else:
            o.append(f"    {dst} = acc;")
        o.append("  }")

    # groups never straddle the L/U boundary
    groups = [(g, min(nl, g + group)) for g in range(0, nl, group)]
    groups += [(g, min(cnt, g + group)) for g in range(nl, cnt, group)]
    for g0, g1 in groups:
        for x in range(g0, g1):
            accumulate(x, f"u[{x - g0}]")
        if g0 == nl:
            o.append("  d = u[0];")
            o.append("  u[0] = (T)1 / u[0];")
        for x in range(g0, g1):
            val = f"l[{x}]" if x < nl else f"u[{x - g0}]"
            o.append(f"  own[{rank[base + x]} * ost] = {val};")
    o.append("  return d;")
    o.append("}")
    o.append("")
    return o


def generate() -> str:
    slots, base, diag, count = slot_tables()
    index = {}
    for c in range(3):
        for s in range(base[c], base[c] + count[c]):
            index[(c,) + slots[s]] = s
    # pivot points of all three row types: the f row's list is the union
    nbrs = []
    for c in (2, 0, 1):
        for s in range(base[c], diag[c]):
            off = slots[s][:4]
            if off not in nbrs:
                nbrs.append(off)
    rank = [slot_rank(s, base, diag, count) for s in range(len(slots))]
    hdr = [
        "// Generated by gen_ilu_rows.py from the KKT row stencils -- do not edit by hand.",
        "// Slot list of the three row types (C, G, f) and their rows in a chunk block.",
        "#pragma once",
        "",
        f"constexpr long long kGenSlotChecksum = {checksum(slots)}LL;",
        f"constexpr int kGenSlots = {len(slots)};",
        f"constexpr int kGenRowSlots0 = {count[0]}, kGenRowSlots1 = {count[1]}, kGenRowSlots2 = {count[2]};",
        "// rank of each slot in a chunk block",
        "constexpr short kGenRank[%d] = {" % len(slots),
    ]
    for a in range(0, len(slots), 20):
        hdr.append("    " + ", ".join(str(r) for r in rank[a:a + 20]) + ",")
    hdr.append("};")
    hdr.append("#ifdef __CUDACC__")
    hdr.append("// per slot: level offset dt, spatial offsets dz, dy, dx and column component")
    hdr.append("__constant__ signed char c_gen_slot[%d][5] = {" % len(slots))
    for a in range(0, len(slots), 8):
        hdr.append("    " + ", ".join("{%d, %d, %d, %d, %d}" % sl for sl in slots[a:a + 8]) + ",")
    hdr.append("};")
    hdr.append("// rank of each slot in a chunk block (device copy of kGenRank)")
    hdr.append("__constant__ short c_gen_rank[%d] = {" % len(slots))
    for a in range(0, len(slots), 20):
        hdr.append("    " + ", ".join(str(r) for r in rank[a:a + 20]) + ",")
    hdr.append("};")
    # inverse table: rank of the slot (row type, dt + 1, spatial offset, column component)
    rank_of = [[[[-1] * 3 for _ in range(27)] for _ in range(3)] for _ in range(3)]
    for c in range(3):
        for s in range(base[c], base[c] + count[c]):
            dt, dz, dy, dx, cc = slots[s]
            rank_of[c][dt + 1][(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)][cc] = rank[s]
    hdr.append("// rank of the slot of row type c with level offset dt, spatial offset")
    hdr.append("// d = (dx+1) + 3 (dy+1) + 9 (dz+1) and column component cc, at [c][dt+1][d][cc];")
    hdr.append("// -1 where the row type has no such slot")
    hdr.append("__constant__ short c_gen_rank_of[3][3][27][3] = {")
    for c in range(3):
        hdr.append("    {")
        for t in range(3):
            hdr.append("        {" + ", ".join("{%d, %d, %d}" % tuple(v) for v in rank_of[c][t]) + "},")
        hdr.append("    },")
    hdr.append("};")
    hdr.append("#endif")
    hdr.append("")
    out = [
        "// Generated by gen_ilu_rows.py from the KKT row stencils -- do not edit by hand.",
        "// ILU(0) elimination of one row of each type (C, G, f), one target entry at a time,",
        "// on the chunk layout (slot s of a point at offset kGenRank[s] * stride).",
        "#pragma once",
        "",
        f"constexpr int kGenNbrs = {len(nbrs)};",
        "// pivot point offsets (dt, dz, dy, dx) shared by the three row types",
        "__constant__ signed char c_gen_nbr[%d][4] = {" % len(nbrs),
        "    " + ", ".join(f"{{{dt}, {dz}, {dy}, {dx}}}" for (dt, dz, dy, dx) in nbrs) + "};",
        "",
    ]
    for c in range(3):
        nl = diag[c] - base[c]
        # contributions to each target entry x of the row, in increasing L-slot order
        contrib = {x: [] for x in range(count[c])}
        for s in range(base[c], diag[c]):
            dt, dz, dy, dx, ck = slots[s]
            i = nbrs.index((dt, dz, dy, dx))
            for t in range(diag[ck] + 1, base[ck] + count[ck]):
                key = (c, dt + slots[t][0], dz + slots[t][1], dy + slots[t][2], dx + slots[t][3], slots[t][4])
                if key in index:
                    x = index[key] - base[c]
                    assert x > s - base[c]
                    contrib[x].append((s - base[c], i, t))
        nupd = sum(len(v) for v in contrib.values())
        out.append(f"// row type {'CGf'[c]}: {count[c]} slots, {nl} L-slots, {nupd} updates")
        out.append(f"constexpr int kGenRowUpdates{c} = {nupd};")
        for prec, gmax in (("32", GROUP32), ("64", GROUP64)):
            out.extend(row_function(c, prec, gmax, nl, count[c], base[c], slots, diag, rank, nbrs, contrib))
    return "\n".join(hdr) + "\n", "\n".join(out) + "\n"


if __name__ == "__main__":
    slots_h, rows = generate()
    for name, text in (("ilu_slots.inc", slots_h), ("ilu_rows.inc", rows)):
        path = os.path.join(HERE, name)
        with open(path, "w") as fh:
            fh.write(text)
        print(path)
