"""The trace summaries on a hand-made timeline (no GPU)."""

import pytest

from paper_2007_03576_gb300 import trace


def test_union_and_overlap_lengths():
    assert trace.union_length([]) == 0.0
    assert trace.union_length([(0, 1), (0.5, 2), (3, 4)]) == pytest.approx(3.0)
    assert trace.union_length([(3, 4), (0, 1), (1, 2)]) == pytest.approx(3.0)
    assert trace.overlap_length([(0, 2)], [(1, 3)]) == pytest.approx(1.0)
    assert trace.overlap_length([(0, 1)], [(1, 2)]) == pytest.approx(0.0)
    assert trace.overlap_length([(0, 4)], [(1, 2), (1.5, 3)]) == pytest.approx(2.0)


def test_summarize_a_small_timeline(tmp_path):
    # one chase step with its side-stream products inside it, then an AED
    # with Z products beside it
    rows = [
        (0, 0, 0.0, 1.0),    # chase
        (2, 1, 0.1, 0.6),    # side products, inside the chase
        (0, 1, 1.0, 1.5),    # main products
        (0, 2, 2.0, 5.0),    # AED
        (1, 5, 2.5, 4.0),    # Z products beside it
    ]
    p = tmp_path / "t.csv"
    p.write_text("stream,phase,start_ms,end_ms\n" + "".join(f"{s},{ph},{a},{b}\n" for s, ph, a, b in rows))
    s = trace.summarize(str(p))
    assert s["rows"] == 5
    assert s["span_ms"] == pytest.approx(5.0)
    assert s["totals_ms"][("main", "chase")] == pytest.approx(1.0)
    assert s["totals_ms"][("side", "products")] == pytest.approx(0.5)
    assert s["totals_ms"][("z", "z_products")] == pytest.approx(1.5)
    assert s["union_ms"]["products"] == pytest.approx(0.5 + 0.5 + 1.5)
    assert s["overlap_ms"][("chase", "side")] == pytest.approx(0.5)
    assert s["overlap_ms"][("aed", "z")] == pytest.approx(1.5)
    assert s["overlap_ms"][("main", "side")] == pytest.approx(0.5)
