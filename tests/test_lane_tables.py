"""The warp-cooperative kernels' lane tables (J = 6) must cover each of the
216 taps exactly once per point and keep every shared-memory instruction free
of bank conflicts for the unpadded tile pitch (E, E^2), E = T + 5."""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1605_05231_gb300", "csrc",
                   "interp_common.cuh")


def _table(name):
    src = open(SRC).read()
    m = re.search(name + r"\[\d+\] = \{([^}]*)\}", src)
    assert m, name
    return [int(v) for v in m.group(1).split(",")]


@pytest.mark.parametrize("E", [13, 21])
def test_lane_tables_cover_taps_and_avoid_bank_conflicts(E):
    main = _table(f"kLaneMain{E}")
    ovf = _table(f"kLaneOvf{E}")
    assert len(main) == 32 and len(ovf) == 24
    taps = []
    for m in main:
        jx, jy = m & 7, (m >> 3) & 7
        taps += [(jx, jy, jz) for jz in range(6)]
    for o in ovf:
        taps.append((o & 7, (o >> 3) & 7, (o >> 6) & 7))
    assert sorted(taps) == sorted((x, y, z) for x in range(6) for y in range(6) for z in range(6))
    # 64-bit accesses: one wavefront per half-warp if the 16 float2 offsets are distinct mod 16
    for jz in range(6):
        for half in (main[:16], main[16:]):
            res = [((m & 7) + E * ((m >> 3) & 7) + E * E * jz) % 16 for m in half]
            assert len(set(res)) == len(res)
    for half in (ovf[:16], ovf[16:]):
        res = [((o & 7) + E * ((o >> 3) & 7) + E * E * ((o >> 6) & 7)) % 16 for o in half]
        assert len(set(res)) == len(res)
