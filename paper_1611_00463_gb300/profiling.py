"""Summaries of Nsight Compute CSV output for this library's kernels.

`python -m paper_1611_00463_gb300.profiling launches <ncu.csv> [--whole-sorts]`
prints, per kernel, the number of launches, the total device time and its
share of a launch list taken with `ncu --metrics gpu__time_duration.sum --csv`;
`--whole-sorts` drops the launches after the last sort's closing statistics
kernel (a list cut off by `ncu -c` mid-sort); `--last-sort` lists the last
whole sort's launches in order instead (each kernel's time and grid).
`python -m paper_1611_00463_gb300.profiling metrics <raw.csv> [regex]` prints
selected metrics of a `ncu -i <rep> --page raw --csv` export, per launch.
"""
from __future__ import annotations

import csv
import io
import re
import sys

SHORT = [("unsigned long", "u64"), ("unsigned int", "u32"), ("bool", "")]


def _csv_rows(path: str) -> list[dict]:
    text = open(path).read().splitlines()
    start = next(i for i, ln in enumerate(text) if ln.startswith('"ID"'))
    return list(csv.DictReader(io.StringIO("\n".join(text[start:]))))


def kernel_label(name: str) -> str:
    m = re.search(r"pgs::(k_\w+)(<[^(]*>)?", name)
    if not m:
        return "other: " + re.sub(r"\(.*", "", name)[-60:]
    label = m.group(1) + (m.group(2) or "")
    for a, b in SHORT:
        label = label.replace(a, b)
    return label.replace(" ", "")


def launches(path: str, whole_sorts: bool = False) -> str:
    rows = [r for r in _csv_rows(path) if r.get("Metric Name") == "gpu__time_duration.sum"]
    if whole_sorts:
        ends = [i for i, r in enumerate(rows) if kernel_label(r["Kernel Name"]) == "k_stats"]
        rows = rows[:ends[-1] + 1] if ends else []
    agg: dict[str, list] = {}
    for r in rows:
        d = agg.setdefault(kernel_label(r["Kernel Name"]), [0, 0.0])
        d[0] += 1
        d[1] += float(r["Metric Value"]) * (1e-3 if r["Metric Unit"] == "ns" else 1.0)
    total = sum(v[1] for v in agg.values())
    out = [f"{'kernel':44s} {'launches':>8s} {'total_us':>12s} {'share':>7s}"]
    for k, (cnt, us) in sorted(agg.items(), key=lambda x: -x[1][1]):
        out.append(f"{k:44s} {cnt:8d} {us:12.1f} {100 * us / total:6.2f}%")
    out.append(f"{'total':44s} {len(rows):8d} {total:12.1f}")
    return "\n".join(out)


def last_sort(path: str) -> str:
    rows = [r for r in _csv_rows(path) if r.get("Metric Name") == "gpu__time_duration.sum"]
    ends = [i for i, r in enumerate(rows) if kernel_label(r["Kernel Name"]) == "k_stats"]
    if not ends:
        return "no whole sort in the list"
    first = ends[-2] + 1 if len(ends) > 1 else 0
    out, total = [], 0.0
    for r in rows[first:ends[-1] + 1]:
        us = float(r["Metric Value"]) * (1e-3 if r["Metric Unit"] == "ns" else 1.0)
        total += us
        out.append(f"{kernel_label(r['Kernel Name']):44s} {us:9.2f} us  grid {r.get('Grid Size', '')}")
    out.append(f"{'total':44s} {total:9.2f} us  {len(out)} launches")
    return "\n".join(out)


def metrics(path: str, pattern: str = r"dram__bytes_(read|write)\.sum$|gpu__time_duration\.sum$|"
                                      r"dram__throughput\.avg\.pct_of_peak_sustained_elapsed|"
                                      r"sm__warps_active\.avg\.pct_of_peak_sustained_active|"
                                      r"launch__registers_per_thread|launch__occupancy_limit") -> str:
    text = open(path).read().splitlines()
    start = next(i for i, ln in enumerate(text) if ln.startswith('"ID"'))
    rows = list(csv.reader(io.StringIO("\n".join(text[start:]))))
    head, units, data = rows[0], rows[1], rows[2:]
    rx = re.compile(pattern)
    cols = [i for i, h in enumerate(head) if rx.search(h)]
    name_col = head.index("Kernel Name")
    out = []
    for row in data:
        out.append(kernel_label(row[name_col]))
        for i in cols:
            out.append(f"  {head[i]} [{units[i]}] = {row[i]}")
    return "\n".join(out)


if __name__ == "__main__":
    if len(sys.argv) < 3 or sys.argv[1] not in ("launches", "metrics"):
        sys.exit(__doc__)
    if sys.argv[1] == "launches" and "--last-sort" in sys.argv[3:]:
        print(last_sort(sys.argv[2]))
    elif sys.argv[1] == "launches":
        print(launches(sys.argv[2], "--whole-sorts" in sys.argv[3:]))
    else:
        print(metrics(sys.argv[2], *sys.argv[3:]))
