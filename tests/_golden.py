"""Readers for the fixtures under tests/golden/ (no arithmetic of the method)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_value(name: str):
    """A value the paper states (tests/golden/paper_values.txt), as int or float."""
    with open(os.path.join(GOLDEN, "paper_values.txt")) as f:
        for line in f:
            fields = line.split("#", 1)[0].split()
            if len(fields) == 2 and fields[0] == name:
                v = fields[1]
                return float(v) if any(c in v for c in ".e") else int(v)
    raise KeyError(name)


def oracle_cases():
    """The stored oracle runs (tests/golden/oracle_runs.txt), one dict per case."""
    cases = []
    with open(os.path.join(GOLDEN, "oracle_runs.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kv = dict(item.split("=", 1) for item in line.split())
            c = {k: int(kv[k]) for k in ("geometry", "boundary", "Lx", "Ly", "n_A", "seed", "mcs", "n_unlike",
                                         "attempts", "unlike", "draws", "accepts")}
            c["omega_over_kT"] = float(kv["omega_over_kT"])
            N = c["Lx"] * c["Ly"]
            bits = np.unpackbits(np.frombuffer(bytes.fromhex(kv["lattice"]), dtype=np.uint8), bitorder="little")
            c["lattice"] = bits[:N].astype(np.uint8)
            hist = [tuple(int(v) for v in p.split(":")) for p in kv["hist_A"].split(",") if p]
            c["hist_A"] = (np.array([s for s, _ in hist], dtype=np.int64), np.array([n for _, n in hist], dtype=np.int64))
            cases.append(c)
    return cases
