"""The tap order of the thread-per-point spread (csrc/spread_taps.inc).

Spread variant 4 runs 32 points per warp whose first-tap offsets differ
modulo 32, visits the taps group by group and synchronises the warp only
between groups.  That is race-free and bank-conflict-free only if every group
holds taps of one offset residue modulo 32 (so lane l's cells in the group are
congruent to its own base offset, distinct from every other lane's) and the
groups together cover the 216 taps exactly once.
"""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1605_05231_gb300", "csrc",
                   "spread_taps.inc")


def _taps(E):
    src = open(SRC).read()
    m = re.search(r"#define NUFFT_SPREAD_TAPS_E%d\(X\)(.*?)(?:\n#define|\Z)" % E, src, re.S)
    assert m, E
    return [tuple(int(v) for v in t) for t in re.findall(r"X\((\d+),(\d+),(\d+),(\d+)\)", m.group(1))]


@pytest.mark.parametrize("E", [13, 21])
def test_groups_share_a_residue_and_cover_every_tap_once(E):
    taps = _taps(E)
    assert sorted((jx, jy, jz) for jx, jy, jz, _ in taps) == sorted(
        (jx, jy, jz) for jx in range(6) for jy in range(6) for jz in range(6))
    assert taps[-1][3] == 1
    groups, cur = [], []
    for jx, jy, jz, end in taps:
        cur.append(jx + E * jy + E * E * jz)
        if end:
            groups.append(cur)
            cur = []
    assert not cur
    residues = [{o % 32 for o in g} for g in groups]
    assert all(len(r) == 1 for r in residues)
    # one group per residue: 32 points with distinct base residues then touch
    # 32 distinct banks at every step of every group
    assert len({next(iter(r)) for r in residues}) == len(groups)
