"""Record the DRAM traffic of the dominant kernel from an ncu capture.

Usage (after an ncu run with --csv and the metrics dram__bytes_read.sum and
dram__bytes_write.sum on the adjoint pass kernel of a case whose states are
larger than L2):

    python -m paper_2603_02804_gb300.record_traffic KEY CSV AMPS "CASE"

KEY names the workload (e.g. hea20), AMPS is the number of amplitudes one
captured launch processes (samples x 2^n), CASE describes the captured case.
The mean of read + write over the captured launches, divided by AMPS, is
stored in dram_traffic.json beside this file with a hash of the kernel
sources; bench.py scales it to its own launches and reports it only while
the sources are unchanged.
"""
from __future__ import annotations

import csv
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "dram_traffic.json")
SOURCES = ("fused.cu", "kernels.h", "capi.cpp", "planner.cpp", "planner.h", "qf_internal.h")


def sources_sha() -> str:
    h = hashlib.sha256()
    for f in SOURCES:
        with open(os.path.join(HERE, "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


_UNIT = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "tbyte": 1e12}


def launch_bytes(csv_path: str) -> list[float]:
    """read + write bytes of every captured launch in an ncu --csv log."""
    with open(csv_path) as f:
        lines = [l for l in f if l.startswith('"')]
    per = {}
    for row in csv.DictReader(lines):
        name = row.get("Metric Name", "")
        if name not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        v = float(row["Metric Value"].replace(",", ""))
        v *= _UNIT.get(row.get("Metric Unit", "byte").lower(), 1.0)
        per[row["ID"]] = per.get(row["ID"], 0.0) + v
    return [per[k] for k in sorted(per, key=int)]


def main(argv):
    key, csv_path, amps, case = argv[1], argv[2], float(argv[3]), argv[4]
    b = launch_bytes(csv_path)
    if not b:
        raise SystemExit("no dram__bytes_* rows in " + csv_path)
    tab = {}
    if os.path.exists(TABLE):
        with open(TABLE) as f:
            tab = json.load(f)
    mean = sum(b) / len(b)
    tab[key] = {"bytes_per_amp": mean / amps, "case": f"{case}; {len(b)} launches, mean {mean / 1e6:.1f} MB",
                "sources_sha": sources_sha()}
    with open(TABLE, "w") as f:
        json.dump(tab, f, indent=1, sort_keys=True)
    print(key, tab[key])


if __name__ == "__main__":
    main(sys.argv)
