"""Summaries of the timeline that schur_hessenberg writes when the
environment variable SCHUR_TRACE=<file> is set.

The file is CSV "stream,phase,start_ms,end_ms", one row per timed bracket of
one reduction.  Streams: 0 main, 1 Z, 2 side.  Phases: 0 chase, 1 products on
H, 2 AED, 3 AED products, 4 small QR, 5 products on Z.

    from paper_2007_03576_gb300 import trace
    s = trace.summarize("trace.csv")
    s["union_ms"]["products"]      # time during which any product ran
    s["overlap_ms"][("chase", "side")]

No GPU is needed to read a trace."""

import csv

STREAMS = {0: "main", 1: "z", 2: "side"}
PHASES = {0: "chase", 1: "products", 2: "aed", 3: "aed_products", 4: "small_qr", 5: "z_products"}


def load(path):
    """Rows of the trace as (stream, phase, start_ms, end_ms) tuples."""
    rows = []
    with open(path) as f:
        for r in csv.DictReader(f):
            rows.append((int(r["stream"]), int(r["phase"]), float(r["start_ms"]), float(r["end_ms"])))
    return rows


def union_length(intervals):
    """Total length of the union of [a, b) intervals."""
    total, cur_a, cur_b = 0.0, None, None
    for a, b in sorted(intervals):
        if cur_b is None or a > cur_b:
            if cur_b is not None:
                total += cur_b - cur_a
            cur_a, cur_b = a, b
        else:
            cur_b = max(cur_b, b)
    if cur_b is not None:
        total += cur_b - cur_a
    return total


def overlap_length(first, second):
    """Length of the intersection of union(first) and union(second)."""
    events = [(a, 0, 1) for a, _ in first] + [(b, 0, -1) for _, b in first]
    events += [(a, 1, 1) for a, _ in second] + [(b, 1, -1) for _, b in second]
    events.sort(key=lambda e: (e[0], -e[2]))
    depth = [0, 0]
    last, total = None, 0.0
    for t, which, step in events:
        if last is not None and depth[0] > 0 and depth[1] > 0:
            total += t - last
        depth[which] += step
        last = t
    return total


def summarize(path_or_rows):
    """Totals per (stream, phase), the span of the trace, the union of each
    group of intervals and the overlaps that the stream layout relies on."""
    rows = load(path_or_rows) if isinstance(path_or_rows, str) else list(path_or_rows)
    groups = {
        "chase": [(a, b) for s, p, a, b in rows if p == 0],
        "aed": [(a, b) for s, p, a, b in rows if p == 2],
        "main": [(a, b) for s, p, a, b in rows if s == 0],
        "side": [(a, b) for s, p, a, b in rows if s == 2],
        "z": [(a, b) for s, p, a, b in rows if s == 1],
        "products": [(a, b) for s, p, a, b in rows if p in (1, 5)],
    }
    totals = {}
    for s, p, a, b in rows:
        key = (STREAMS.get(s, str(s)), PHASES.get(p, str(p)))
        totals[key] = totals.get(key, 0.0) + (b - a)
    span = (max(b for _, _, _, b in rows) - min(a for _, _, a, _ in rows)) if rows else 0.0
    pairs = [("chase", "side"), ("aed", "z"), ("main", "z"), ("main", "side")]
    return {
        "rows": len(rows),
        "span_ms": span,
        "totals_ms": totals,
        "union_ms": {k: union_length(v) for k, v in groups.items()},
        "overlap_ms": {pair: overlap_length(groups[pair[0]], groups[pair[1]]) for pair in pairs},
    }
