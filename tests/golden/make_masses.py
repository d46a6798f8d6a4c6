"""Write tests/golden/masses.json: the bare masses m0 of the synthetic workloads.

Calls only the oracle.  Reading (the configured bisection has no crossing on
these fields): m0 = 1e-3 - min Re lambda(D(0)) on the 8^4 tuning field, which
puts the left edge of the spectrum of D(m0) at Re = 1e-3.

  8^4, eps = 0.3, csw = 0, seed 0   -> m0 of the two-level FP64 workload
  8^4, eps = 0.4, csw = 1, seed 0   -> m0 reused on 16^3x32 and larger lattices
  8^4, eps = 0.45, csw = 1, seed 0  -> m0 reused on the four-level 48^3x96 lattice
  8^4, eps = 0.8, csw = 1, seed 0   -> rougher fields whose spectrum edge is nearly real (the
                                       near-critical mass scan)

Entries already in masses.json are kept (ARPACK starts from a random vector, so a recomputation
could move the last digits); only missing ones are computed.

Usage: python tests/golden/make_masses.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle.spectrum import edge_mass  # noqa: E402
from oracle.wilson import WilsonOp  # noqa: E402


def main():
    out = {"reading": "m0 = 1e-3 - min Re lambda(D(0)) on an 8^4 field (seed 0), antiperiodic time",
           "masses": {}}
    path = os.path.join(HERE, "masses.json")
    if os.path.exists(path):
        with open(path) as f:
            out["masses"] = json.load(f)["masses"]
    for name, eps, csw in (("eps0.3_csw0", 0.3, 0.0), ("eps0.4_csw1", 0.4, 1.0), ("eps0.45_csw1", 0.45, 1.0),
                           ("eps0.8_csw1", 0.8, 1.0)):
        if name in out["masses"]:
            continue
        U = synth.su3_field((8, 8, 8, 8), eps, 0)
        m0, w = edge_mass(U, csw, -1, margin=1e-3)
        out["masses"][name] = {
            "eps": eps, "csw": csw, "m0": m0,
            "leftmost_eigenvalues_D0": [[float(z.real), float(z.imag)] for z in w[:6]],
        }
        print(name, m0, w[:4])
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
