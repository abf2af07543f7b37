"""Writes tests/golden/oracle_runs.txt: short runs of the oracle (and nothing else)
from its own random start, stored so that the CUDA path can be checked against
them without running the oracle, and so that any later change to the oracle's
arithmetic shows up as a diff of this file.

    python tests/golden/make_oracle_runs.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402

# geometry, boundary, Lx, Ly, n_A, omega/kT, seed, MCS: both geometries, both signs of
# omega, a ragged word tail, a lattice of one word row, the 64x64 workload's shape,
# and the helical seven-colour schedule.
CASES = [
    (oracle.TRI6, oracle.PERIODIC, 24, 20, 200, 0.7, 11, 30),
    (oracle.SQ4, oracle.PERIODIC, 24, 20, 240, -0.5, 12, 30),
    (oracle.TRI6, oracle.PERIODIC, 33, 17, 190, 1.1, 13, 25),
    (oracle.SQ4, oracle.PERIODIC, 7, 9, 30, 0.9, 14, 40),
    (oracle.TRI6, oracle.PERIODIC, 64, 64, 2048, 0.6, 1, 20),
    (oracle.TRI6, oracle.HELICAL, 10, 7, 35, 0.8, 15, 40),
    (oracle.TRI6, oracle.HELICAL, 31, 14, 150, -0.4, 16, 20),
]


def main():
    lines = ["# Oracle runs from the oracle's own start (exactly n_A A sites placed from the seed).",
             "# lattice: site i is bit i % 8 of byte i // 8 (hex); hist_A: size:count of the A clusters.",
             "# Written by tests/golden/make_oracle_runs.py, which calls only oracle/."]
    for g, b, Lx, Ly, nA, bw, seed, mcs in CASES:
        t0 = oracle.init(Lx, Ly, nA, seed)
        if b == oracle.HELICAL:
            r = oracle.run_mpkk(Lx, Ly, bw, seed, t0, 0, mcs)
        else:
            r = oracle.run(Lx, Ly, g, bw, seed, t0, 0, mcs)
        sizes, counts = oracle.cluster_histogram(Lx, Ly, g, r.lattice, 1, b)
        hexlat = np.packbits(r.lattice.astype(np.uint8), bitorder="little").tobytes().hex()
        hist = ",".join(f"{s}:{c}" for s, c in zip(sizes.tolist(), counts.tolist()))
        lines.append(f"geometry={g} boundary={b} Lx={Lx} Ly={Ly} n_A={nA} omega_over_kT={bw!r} seed={seed} "
                     f"mcs={mcs} n_unlike={r.n_unlike} attempts={r.attempts} unlike={r.unlike} draws={r.draws} "
                     f"accepts={r.accepts} hist_A={hist} lattice={hexlat}")
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_runs.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
