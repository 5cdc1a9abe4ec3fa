"""Per-kernel summary of an ncu launch list (--metrics gpu__time_duration.sum --csv): launches,
total device time and share.  Usage: python ncu_launch_summary.py launches.csv [skip_kernel ...]
(kernels whose names start with a prefix given after the file are reported but left out of
the shares, e.g. the input generator)."""
import collections
import csv
import re
import sys


def short_name(full):
    name = full.replace("<unnamed>::", "").replace("(anonymous namespace)::", "")
    name = re.sub(r"^void ", "", name)
    name = name.split("(")[0]
    return name.split("::")[-1]


def main(path, skip=()):
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hi]
    ki, mi, ui, vi = (hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Unit", "Metric Value"))
    scale = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0}
    tot = collections.defaultdict(float)
    cnt = collections.Counter()
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        n = short_name(r[ki])
        tot[n] += float(r[vi].replace(",", "")) * scale.get(r[ui], 1.0)
        cnt[n] += 1
    skipped = lambda k: any(k.startswith(x) for x in skip)
    total = sum(v for k, v in tot.items() if not skipped(k))
    print("| kernel | launches | total ms | share |")
    print("|---|---|---|---|")
    for k, v in sorted(tot.items(), key=lambda kv: -kv[1]):
        share = "-" if skipped(k) else "%.1f%%" % (100 * v / total)
        print("| %s | %d | %.1f | %s |" % (k, cnt[k], v, share))
    print("| total (shares) | %d | %.1f | 100%% |" % (sum(c for k, c in cnt.items() if not skipped(k)), total))


if __name__ == "__main__":
    main(sys.argv[1], tuple(sys.argv[2:]))
