#!/usr/bin/env python
"""Writes tests/golden/energy_ensemble.txt: the oracle's energy errors |dE/E| over ensembles
of rounding-level perturbed starts, for the two configurations whose oracle runs take
minutes (so the GPU tests read them instead of re-running the oracle):

  c2  Plummer 2048 + central SMBH binary (N = 2050), eta = 1e-12, 200 accepted GBS steps
      towards t_end = 10;
  c5  Plummer 10^4 + two SMBHs (N = 10002), eta = 1e-12, 20 accepted GBS steps towards
      t_end = 1 (the first step is ds = q U dt with dt = 1, as in the benchmark).

Realisation k uses workloads.perturbed(..., k): 0 is the unperturbed start, k > 0 scales
every coordinate by 1 + 1e-15 (2u - 1). Only the oracle and the input generators run here.

    python tests/golden/make_energy_ensemble.py [--threads T] [--k K] [--which c2,c5]
"""
from __future__ import annotations

import argparse
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2001_03180_gb300 import workloads as W  # noqa: E402

CONFIGS = {
    "c2": ("plummer2048_smbh_binary", 10.0, 200),
    "c5": ("plummer10k_two_smbh", 1.0, 20),
}
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "energy_ensemble.txt")


def run(name, t_end, steps, k):
    m, r, v = W.perturbed(*W.workload(name), k)
    o = O.System(m, r, v)
    e0 = o.energy()["E"]
    rc, st = o.integrate(t_end, steps)
    e1 = o.energy()["E"]
    return rc, st, abs((e1 - e0) / e0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--which", default="c2,c5")
    a = ap.parse_args()
    O.set_threads(a.threads)
    lines = ["# The oracle's |dE/E| over ensembles of perturbed starts (realisation k: every coordinate",
             "# scaled by 1 + 1e-15 (2u - 1), u from stream (7919, k); k = 0 unperturbed).",
             "# Written by tests/golden/make_energy_ensemble.py, which runs only oracle/ and the input",
             f"# generators; host {platform.machine()} {platform.processor() or ''}, {a.threads} threads.",
             "# Keys: <config>_dE_r<k> |dE/E|, <config>_t_r<k> time reached, <config>_rej_r<k> rejections."]
    for key in a.which.split(","):
        name, t_end, steps = CONFIGS[key]
        lines.append(f"# {key}: {name}, {steps} accepted GBS steps towards t_end = {t_end}, eta = 1e-12")
        for k in range(a.k):
            t0 = time.time()
            rc, st, dE = run(name, t_end, steps, k)
            assert rc == 0 and st["accepted"] == steps, (key, k, rc, st)
            lines += [f"{key}_dE_r{k} {dE:.17g}", f"{key}_t_r{k} {st['t']:.17g}", f"{key}_rej_r{k} {st['rejected']}"]
            print(key, k, dE, st["t"], st["rejected"], f"{time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
