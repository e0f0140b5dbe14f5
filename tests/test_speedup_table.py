"""The shipped F_W table (Sec. 5.B: throughput scaling of packing W over the
conventional inner kernel, measured offline on GB300) and its loading."""
import re

import pytest


def test_shipped_table_is_consistent():
    from paper_1110_5765_gb300 import api
    tab = api.load_speedups()
    assert tab, "f_table.json missing"
    for key, v in tab.items():
        m = re.fullmatch(r"(f32|f64)/sym/W([234])/L(\d+)", key)
        assert m, key
        assert v["F"] == pytest.approx(v["t_conventional_ms"] / v["t_packed_ms"], rel=1e-3)
        assert 1.0 < v["F"] <= int(m.group(2)) + 0.5       # at most about W times faster
    for w in (2, 3, 4):
        assert f"f32/sym/W{w}/L128" in tab and f"f64/sym/W{w}/L64" in tab
    # more packing is faster, and so is a longer slab (fewer unpacks per FMA)
    for dt, L in (("f32", 128), ("f64", 64)):
        Fs = [tab[f"{dt}/sym/W{w}/L{L}"]["F"] for w in (2, 3, 4)]
        assert Fs == sorted(Fs)
