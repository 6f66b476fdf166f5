"""Summarises an ncu launch list (CSV of gpu__time_duration.sum per launch) into per-kernel
launches, total time and share.  Usage: python -m paper_2109_13628_gb300.ncu_summary launches.csv"""
import collections
import csv
import re
import sys


def summarise(path):
    rows = list(csv.reader(open(path)))
    hdr_i = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hdr_i]
    ki, mi, vi, ui = hdr.index("Kernel Name"), hdr.index("Metric Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hdr_i + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}.get(r[ui], 1.0)
        name = re.sub(r"\(.*", "", r[ki])
        agg[name][0] += 1
        agg[name][1] += float(r[vi].replace(",", "")) * scale
    return agg


def main(path):
    agg = summarise(path)
    tot = sum(a[1] for a in agg.values())
    print(f"| kernel | launches | total us | avg us | share |\n|---|---:|---:|---:|---:|")
    for name, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"| `{name}` | {n} | {t:.1f} | {t / n:.2f} | {t / tot:.3f} |")
    print(f"\ntotal {tot:.1f} us over {sum(a[0] for a in agg.values())} launches")


if __name__ == "__main__":
    main(sys.argv[1])
