"""Summarise an ncu CSV launch list (``--metrics gpu__time_duration.sum --csv``):
per kernel its launches, total device time and share.  Usage:
    python -m paper_1804_07017_gb300.ncu_summary launches.csv
"""
from __future__ import annotations

import collections
import csv
import re
import sys


def short_name(name: str) -> str:
    name = re.sub(r"\(.*$", "", name)            # drop the argument list
    name = name.replace("<unnamed>::", "")
    name = re.sub(r"^void\s+", "", name)
    return name.strip()


def summarise(path: str):
    with open(path) as f:
        lines = [ln for ln in f if not ln.startswith("==")]
    agg = collections.defaultdict(lambda: [0, 0.0])
    scale = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0}
    for row in csv.DictReader(lines):
        if row.get("Metric Name") != "gpu__time_duration.sum":
            continue
        v = float(row["Metric Value"].replace(",", "")) * scale.get(row["Metric Unit"], 1e-6)
        k = short_name(row["Kernel Name"])
        agg[k][0] += 1
        agg[k][1] += v
    total = sum(v[1] for v in agg.values())
    out = []
    for k, (cnt, ms) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append((k, cnt, ms, ms / total if total else 0.0))
    return out, total


if __name__ == "__main__":
    rows, total = summarise(sys.argv[1])
    print(f"{'kernel':60s} {'launches':>8s} {'total ms':>10s} {'share':>7s}")
    for k, cnt, ms, sh in rows:
        print(f"{k:60s} {cnt:8d} {ms:10.3f} {100 * sh:6.1f}%")
    print(f"{'total':60s} {sum(r[1] for r in rows):8d} {total:10.3f}")
