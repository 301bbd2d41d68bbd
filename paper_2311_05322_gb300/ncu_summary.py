"""Summarise an ncu launch list (``--metrics gpu__time_duration.sum --csv``) per kernel.

Prints a markdown table of launches, total and mean device time and share, separately for the
setup kernels (geometry, subdomain factorisation and packing) and the solve-phase kernels that
make up each bench step.  Usage: python -m paper_2311_05322_gb300.ncu_summary launches.csv
"""
from __future__ import annotations

import csv
import re
import sys
from collections import defaultdict

SETUP = ("elem_geom", "face_geom", "tikhonov_weights", "local_assemble", "gj_", "extract_owned", "pack_w",
         "fill_pattern",  # fill_pattern: timing inputs of the launch-shape tuner
         "port_face", "port_accumulate", "port_norm",  # port load vectors (once per boundary)
         "mf_assemble", "mf_extend_add", "mf_extract")  # sparse subdomain factorisation


def short(name: str) -> str:
    m = re.search(r"([A-Za-z0-9_]+_kernel)(<[^()]*>)?", name)
    if not m:
        return name[:60]
    return m.group(1) + (m.group(2) or "")


def summarise(path: str) -> str:
    rows = []
    with open(path) as f:
        lines = [l for l in f if l.startswith('"')]
    for r in csv.DictReader(lines):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        rows.append((short(r["Kernel Name"]), float(r["Metric Value"]) * (1e-3 if r["Metric Unit"] == "ns" else 1.0)))
    out = []
    for title, pick in (("solve phase (per-step kernels)", lambda k: not k.startswith(SETUP)),
                        ("setup (once per mesh / preconditioner)", lambda k: k.startswith(SETUP))):
        agg = defaultdict(lambda: [0, 0.0])
        for k, us in rows:
            if pick(k):
                agg[k][0] += 1
                agg[k][1] += us
        tot = sum(v[1] for v in agg.values())
        out.append(f"### {title}: {sum(v[0] for v in agg.values())} launches, {tot / 1e3:.1f} ms\n")
        out.append("| kernel | launches | total ms | mean us | share |")
        out.append("|---|---:|---:|---:|---:|")
        for k, (n, us) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
            out.append(f"| `{k}` | {n} | {us / 1e3:.2f} | {us / n:.1f} | {100 * us / tot:.1f}% |")
        out.append("")
    return "\n".join(out)


if __name__ == "__main__":
    print(summarise(sys.argv[1]))
