"""Summarize an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel: launches, total time, share."""
import csv
import re
import sys
from collections import defaultdict


def main(path, skip_prefix=None):
    rows = list(csv.reader(open(path)))
    hdr_i = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hdr_i]
    k_i, m_i, v_i, u_i = hdr.index("Kernel Name"), hdr.index("Metric Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    tot = defaultdict(float)
    cnt = defaultdict(int)
    for r in rows[hdr_i + 1:]:
        if len(r) <= v_i or r[m_i] != "gpu__time_duration.sum":
            continue
        name = re.sub(r"\(.*", "", r[k_i]).strip()
        val = float(r[v_i].replace(",", ""))
        scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}[r[u_i]]
        tot[name] += val * scale
        cnt[name] += 1
    total = sum(tot.values())
    print(f"{'kernel':<60} {'launches':>8} {'total_us':>12} {'share':>7}")
    for name, t in sorted(tot.items(), key=lambda kv: -kv[1]):
        print(f"{name[:60]:<60} {cnt[name]:>8} {t:>12.1f} {100 * t / total:>6.2f}%")
    print(f"{'TOTAL':<60} {sum(cnt.values()):>8} {total:>12.1f}")


if __name__ == "__main__":
    main(sys.argv[1])
