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


def test_fixed_point_lane_tables_cover_taps_and_avoid_bank_conflicts():
    """Spread variant 5 updates 4-byte cells: an instruction is one wavefront
    when its lanes hit distinct banks (offsets distinct mod 32).  Lanes 0..30
    serve one (jx, jy) column each for every jz, lanes 0..29 one more tap;
    255 / 65535 mark a lane without one."""
    E = 13
    main = _table("kLaneMainI13")
    ovf = _table("kLaneOvfI13")
    assert len(main) == 32 and len(ovf) == 32
    assert main[31] == 255 and all(m != 255 for m in main[:31])
    assert ovf[30:] == [65535, 65535] and all(o != 65535 for o in ovf[:30])
    taps = []
    for m in main[:31]:
        taps += [(m & 7, (m >> 3) & 7, jz) for jz in range(6)]
    taps += [(o & 7, (o >> 3) & 7, (o >> 6) & 7) for o in ovf[:30]]
    assert sorted(taps) == sorted((x, y, z) for x in range(6) for y in range(6) for z in range(6))
    for jz in range(6):
        res = [((m & 7) + E * ((m >> 3) & 7) + E * E * jz) % 32 for m in main[:31]]
        assert len(set(res)) == 31
    for group in (ovf[:15], ovf[15:30]):
        res = [((o & 7) + E * ((o >> 3) & 7) + E * E * ((o >> 6) & 7)) % 32 for o in group]
        assert len(set(res)) == len(res)


def test_fixed_point_pad_lanes_take_free_banks():
    """Lanes without a tap of their own add zero at a cell whose bank is free
    in their instruction: the main instructions reach 32 distinct banks, the
    extra-tap instruction at most two lanes per bank."""
    E = 13
    main = _table("kLaneMainI13")
    ovf = _table("kLaneOvfI13")
    pad = _table("kPadI13")
    assert len(pad) == 3
    for jz in range(6):
        res = [((m & 7) + E * ((m >> 3) & 7) + E * E * jz) % 32 for m in main[:31]] + [(pad[0] + E * E * jz) % 32]
        assert len(set(res)) == 32
    res = [((o & 7) + E * ((o >> 3) & 7) + E * E * ((o >> 6) & 7)) % 32 for o in ovf[:30]] + [pad[1] % 32, pad[2] % 32]
    assert max(res.count(r) for r in set(res)) <= 2
    # every pad cell stays inside the 13^3 plane for any tile offset of an 8^3 tile
    top = 7 * E * E + 7 * E + 7
    assert top + pad[0] + 5 * E * E < E ** 3 and top + max(pad[1:]) < E ** 3
