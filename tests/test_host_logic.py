"""Host-side logic without a GPU: the key mapping between the oracle's hit records and
the C ABI's hit keys (every encoding: mesh segments, the two cross terms, point routes,
point route pairs, water-column scatterers), and the bench's reading of the committed
profile counters (used only while the kernel's source matches the capture)."""
import hashlib
import os

import numpy as np

from tests import parity

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _hits(rows):
    cols = list(zip(*rows))
    return {"ray": np.array(cols[0], np.int32), "sub": np.array(cols[1], np.int32),
            "seg": np.array(cols[2], np.int32), "prim": np.array(cols[3], np.int32)}


def test_oracle_keys_cover_every_hit_kind():
    n_sub = 4
    h = _hits([
        (7, 3, 0, 11),                   # mesh, direct
        (7, 3, 1, 12),                   # mesh, one bounce
        (7, 3, 1 | 16, 12),              # cross term returning straight
        (7, 3, 1 | 32, 12),              # cross term returning along the route
        (2, 1, 1, -1),                   # point 2, route 1
        (2, 0x10000 | (1 << 8) | 2, 2, -1),  # point 2, out route 1, back route 2
        (123456, 0x20000, 0, -1),        # water-column scatterer 123456
    ])
    k = parity.oracle_keys(h, n_sub)
    sr = 7 * n_sub + 3
    want = [sr << 2, (sr << 2) | 1, (sr << 2) | 1 | 0x40000000, (sr << 2) | 1 | 0x20000000,
            0x80000000 | (2 << 8) | 1, 0xC0000000 | (2 << 16) | (1 << 8) | 2, 0xA0000000 | 123456]
    assert [int(x) for x in k] == want
    assert len(set(int(x) for x in k)) == len(want)


def test_profile_counters_follow_the_source_hash():
    import bench
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    rows = {l.split()[0]: l.split() for l in open(path) if l.strip() and not l.startswith("#")}
    src = hashlib.sha1(open(os.path.join(ROOT, "paper_2606_06130_gb300", "csrc", "synth_tc.cu"), "rb")
                       .read()).hexdigest()[:12]
    traffic, inst = bench.read_profile("k_synth_tz")
    if rows["k_synth_tz"][2] == src:
        assert traffic == float(rows["k_synth_tz"][1]) and inst == float(rows["k_synth_tz"][3])
    else:
        assert traffic is None and inst is None
    assert bench.read_profile("k_no_such_kernel") == (None, None)
