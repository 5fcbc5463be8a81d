"""Host checks of the generated slot tables that the factorisation kernels index.

* Regenerating ilu_slots.inc and ilu_rows.inc reproduces the committed files.
* The inverse table c_gen_rank_of agrees with the slot list (c_gen_slot,
  c_gen_rank), and the slots that the value gather writes -- per spatial
  offset: C row C and f columns at levels n-1, n; G row G column at n, n+1;
  f row G and f columns at n-1, n, n+1; the G row's two sensor slots at the
  centre -- hit every chunk-block rank exactly once and never a -1 entry
  (which would be an out-of-range store).
"""

import importlib.util
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1508_06103_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_ilu_rows", os.path.join(CSRC, "gen_ilu_rows.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _table(text, name):
    body = text[text.index(name):]
    body = body[body.index("= {") + 3:body.index("};")]
    return [int(v) for v in re.findall(r"-?\d+", body)]


def test_generated_files_are_current():
    slots_h, rows = _gen().generate()
    with open(os.path.join(CSRC, "ilu_slots.inc")) as fh:
        assert fh.read() == slots_h
    with open(os.path.join(CSRC, "ilu_rows.inc")) as fh:
        assert fh.read() == rows


def test_rank_of_matches_slot_list_and_gather_pattern():
    with open(os.path.join(CSRC, "ilu_slots.inc")) as fh:
        text = fh.read()
    slot = _table(text, "c_gen_slot[")
    rank = _table(text, "c_gen_rank[")
    rank_of = _table(text, "c_gen_rank_of[")
    ns = len(rank)
    assert ns == 326 and len(slot) == 5 * ns and len(rank_of) == 3 * 3 * 27 * 3
    counts = (108, 56, 162)

    def r_of(c, dt, d, cc):
        return rank_of[((c * 3 + dt + 1) * 27 + d) * 3 + cc]

    s = 0
    for c in range(3):
        for _ in range(counts[c]):
            dt, dz, dy, dx, cc = slot[5 * s:5 * s + 5]
            assert r_of(c, dt, (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1), cc) == rank[s]
            s += 1
    assert sum(v >= 0 for v in rank_of) == ns

    written = []
    for d in range(27):
        written += [(0, 0, d, 0), (0, 0, d, 2), (0, -1, d, 0), (0, -1, d, 2), (1, 0, d, 1), (1, 1, d, 1)]
        if d == 13:
            written += [(1, 0, d, 0), (1, 1, d, 0)]
        written += [(2, dt, d, cc) for dt in (-1, 0, 1) for cc in (1, 2)]
    ranks = [r_of(*k) for k in written]
    assert min(ranks) >= 0
    assert sorted(ranks) == list(range(ns))
