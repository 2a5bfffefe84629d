"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv):
per kernel the launch count, total device time and share.  Usage:
    python profiles/summarize_launches.py launches.csv [regex-of-interest]
"""
import collections
import csv
import re
import sys


def short(name):
    name = re.sub(r"\(.*", "", name)
    name = re.sub(r"^void ", "", name)
    name = re.sub(r"<.*", "", name) if "srn::" not in name else name
    for k in ["render_mma_kernel", "render_fp32_kernel", "dvr_dense_kernel", "eval_fp32_kernel", "fit_point_kernel",
              "sort_hist_kernel", "sort_scatter_kernel", "scan_kernel", "cell_start_kernel", "grid_grad_kernel",
              "reduce_parts_kernel", "adam_kernel", "to_half_kernel", "mse_kernel", "mse1_kernel",
              "gauss_pass_kernel", "resample_kernel"]:
        if k in name:
            return "srn::" + k
    return name[:60]


def main(path):
    rows = [r for r in csv.DictReader(l for l in open(path) if not l.startswith("=="))
            if r["Metric Name"] == "gpu__time_duration.sum"]
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows:
        v = float(r["Metric Value"].replace(",", ""))
        unit = r["Metric Unit"]
        ns = v * {"nsecond": 1, "usecond": 1e3, "msecond": 1e6, "second": 1e9}.get(unit, 1)
        a = agg[short(r["Kernel Name"])]
        a[0] += 1
        a[1] += ns
    tot = sum(v[1] for v in agg.values())
    print(f"{'kernel':44s} {'launches':>8s} {'total ms':>10s} {'share':>7s}")
    for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"{k:44s} {n:8d} {t / 1e6:10.3f} {100 * t / tot:6.2f}%")
    print(f"{'all':44s} {sum(v[0] for v in agg.values()):8d} {tot / 1e6:10.3f}")


if __name__ == "__main__":
    main(sys.argv[1])
