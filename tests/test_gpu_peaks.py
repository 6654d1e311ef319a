"""The arithmetic-unit probes that give bench.py's roofline denominators."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_peak_probes_run_and_report():
    import paper_1403_0555_b300 as gb
    v = {k: gb.gc_peak_probe(getattr(gb, k)) for k in
         ("GC_PEAK_FFMA", "GC_PEAK_FFMA2", "GC_PEAK_DFMA", "GC_PEAK_RSQ", "GC_PEAK_DFMA_LANE1")}
    print("\n" + ", ".join(f"{k[8:]} {x / 1e12:.3f} T/s" for k, x in v.items()))
    assert all(math.isfinite(x) and x > 0 for x in v.values())
    # FP32 is the fast unit on every part this library targets
    assert v["GC_PEAK_FFMA"] > 10 * v["GC_PEAK_DFMA"]
    with pytest.raises(gb.GribovError) as e:
        gb.gc_peak_probe(17)
    assert e.value.code == gb.GC_EINVAL
