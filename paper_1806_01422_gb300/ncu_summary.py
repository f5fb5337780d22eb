"""Summaries of ncu output for the profiles/ folder (reads ncu files; runs no GPU code).

    python -m paper_1806_01422_gb300.ncu_summary launches FILE.csv
        per kernel: launches, total device time and share (from a
        `--metrics gpu__time_duration.sum --csv --log-file` capture)
    python -m paper_1806_01422_gb300.ncu_summary report FILE.ncu-rep
        per captured launch: duration, DRAM bytes, pipe utilisation, warps,
        registers and the main stall reasons (needs the `ncu` CLI to export)
    python -m paper_1806_01422_gb300.ncu_summary raw FILE.csv
        the same from `ncu -i FILE.ncu-rep --page raw --csv` output
"""
import collections
import csv
import io
import subprocess
import sys

KEYS = [
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput % of peak"),
    ("sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active", "FP64 pipe % active"),
    ("sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", "FMA (FP32) pipe % active"),
    ("sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active", "ALU pipe % active"),
    ("sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active", "LSU pipe % active"),
    ("sm__throughput.avg.pct_of_peak_sustained_elapsed", "SM throughput % of peak"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active % of peak"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue active %"),
    ("launch__registers_per_thread", "registers/thread"),
    ("launch__grid_size", "grid"),
    ("launch__block_size", "block"),
    ("launch__shared_mem_per_block_dynamic", "dynamic smem/block"),
    ("smsp__average_warps_issue_stalled_wait_per_issue_active.ratio", "stall: wait"),
    ("smsp__average_warps_issue_stalled_short_scoreboard_per_issue_active.ratio", "stall: short scoreboard"),
    ("smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio", "stall: long scoreboard"),
    ("smsp__average_warps_issue_stalled_barrier_per_issue_active.ratio", "stall: barrier"),
    ("smsp__average_warps_issue_stalled_math_pipe_throttle_per_issue_active.ratio", "stall: math pipe throttle"),
]


def launches(path):
    rows = list(csv.reader(open(path)))
    hi = [i for i, r in enumerate(rows) if "Kernel Name" in r][0]
    h = rows[hi]
    ki, mi, vi, ui = h.index("Kernel Name"), h.index("Metric Name"), h.index("Metric Value"), h.index("Metric Unit")
    agg = collections.OrderedDict()
    unit = None
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = r[ki].split("(")[0].replace("void ", "")
        unit = r[ui]
        n, t = agg.get(name, (0, 0.0))
        agg[name] = (n + 1, t + float(r[vi].replace(",", "")))
    tot = sum(t for _, t in agg.values())
    out = ["| kernel | launches | total (%s) | share |" % unit, "|---|---|---|---|"]
    for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append("| `%s` | %d | %.1f | %.3f |" % (k, n, t, t / tot))
    out.append("| all | %d | %.1f | 1.000 |" % (sum(n for n, _ in agg.values()), tot))
    return "\n".join(out)


def report(path, raw=None):
    if raw is None:
        raw = subprocess.run(["ncu", "-i", path, "--page", "raw", "--csv"], capture_output=True, text=True,
                             check=True).stdout
    rows = list(csv.reader(io.StringIO(raw)))
    h, units = rows[0], rows[1]
    out = []
    for r in rows[2:]:
        out.append("### `%s`" % r[h.index("Kernel Name")].split("(")[0].replace("void ", ""))
        out.append("")
        out.append("| metric | value |")
        out.append("|---|---|")
        for key, label in KEYS:
            if key in h:
                i = h.index(key)
                out.append("| %s | %s %s |" % (label, r[i], units[i]))
        out.append("")
    return "\n".join(out)


if __name__ == "__main__":
    kind, path = sys.argv[1], sys.argv[2]
    if kind == "launches":
        print(launches(path))
    elif kind == "raw":
        print(report(None, raw=open(path).read()))
    else:
        print(report(path))
