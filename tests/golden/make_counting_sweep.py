#!/usr/bin/env python
"""Writes counting_sweep_counts.json: FP64 oracle vertex and edge counts of the
counting-sweep nets (Section 5.1.2: four hidden layers of width 10, 20 or 40
and a scalar output, randomly initialised, on [-1,1]^D, five nets per point).

Only the oracle computes these values.  Per width, D runs up to MAX_DIM (the
oracle needs up to 10 minutes for one net at D = 5, width 40, 3 minutes at
D = 6, width 20 and 5 minutes at D = 10, width 10; the next dimension of
the wider nets would take hours and more host memory than a workstation
has); a point is left out when one of its extractions takes longer than
--max-seconds.

  python tests/golden/make_counting_sweep.py [--max-seconds 600] [--only 5:40 ...]

--only recomputes the listed D:width points and merges them into the
existing file.
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2306_07212_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(HERE, "counting_sweep_counts.json")
MAX_DIM = {10: 10, 20: 6, 40: 5}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--max-seconds", type=float, default=600.0)
    ap.add_argument("--only", nargs="*", default=None, help="D:width points to recompute and merge")
    args = ap.parse_args()
    only = None if args.only is None else {tuple(int(x) for x in p.split(":")) for p in args.only}
    points = []
    for width in wl.COUNTING_WIDTHS:
        for D in wl.COUNTING_DIMS:
            if D > MAX_DIM[width]:
                break
            if only is not None and (D, width) not in only:
                continue
            rows, slow = [], False
            for seed in range(wl.COUNTING_SEEDS):
                net, box = wl.counting_sweep_net(D, width, seed)
                t0 = time.perf_counter()
                r = oracle.extract(net, box)
                dt = time.perf_counter() - t0
                if r.status != 0:
                    raise SystemExit(f"oracle status {r.status} at D={D} width={width} seed={seed}: {r.error}")
                rows.append({"seed": seed, "nV": int(r.nV), "nE": int(r.nE)})
                print(f"D={D} width={width} seed={seed}: {r.nV} V {r.nE} E in {dt:.2f} s", flush=True)
                if dt > args.max_seconds:
                    slow = True
                    break
            if slow:
                break  # larger D at this width only takes longer
            points.append({"D": D, "width": width, "counts": rows})
    if only is not None:
        with open(OUT) as f:
            kept = [p for p in json.load(f)["points"] if (p["D"], p["width"]) not in only]
        points = sorted(kept + points, key=lambda p: (wl.COUNTING_WIDTHS.index(p["width"]), p["D"]))
    doc = {"source": "FP64 oracle (oracle/) on paper_2306_07212_gb300.workloads.counting_sweep_net; "
                     "written by tests/golden/make_counting_sweep.py",
           "box": "[-1,1]^D", "network": "[D, w, w, w, w, 1], uniform +-1/sqrt(fan_in), rounded to FP32",
           "points": points}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
