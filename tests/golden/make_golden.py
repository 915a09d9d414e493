"""Writes the oracle's golden fixtures (run from the repository root).

Calls only oracle/.  The paper prints no worked example to store, so these
fixtures record the FP64 oracle's own results on fixed seeded inputs; the
tests require every machine to reproduce them bit for bit (the oracle is
built with -ffp-contract=off for exactly that).

  config1_oracle.json: d = 4 symmetric Gaussian (a = 0.1), 50 bins, 1e5
  samples, 5 iterations, alpha = 1.5, seed 0 -- the per-iteration estimates
  and sigmas (as hex floats), the combination, and a SHA-256 of the final
  grid's FP64 bytes.
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402


def config1():
    r = O.integrate(4, 50, "gauss_sym", [0.1], 100_000, 5, alpha=1.5, seed=0)
    return {
        "source": "oracle.integrate(4, 50, 'gauss_sym', [0.1], 100000, 5, alpha=1.5, seed=0)",
        "iters": [[float(I).hex(), float(s).hex()] for I, s in r["iters"]],
        "I": float(r["I"]).hex(), "sigma": float(r["sigma"]).hex(),
        "chi2_dof": float(r["chi2_dof"]).hex(),
        "edges_sha256": hashlib.sha256(r["edges"].astype("<f8").tobytes()).hexdigest(),
    }


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "config1_oracle.json"), "w") as f:
        json.dump(config1(), f, indent=1)
        f.write("\n")
