"""Writes the oracle's golden fixtures (run from the repository root).

Calls only oracle/.  The paper prints no worked example to store, so these
fixtures record the FP64 oracle's own results on fixed seeded inputs; the
tests require every machine to reproduce them bit for bit (the oracle is
built with -ffp-contract=off for exactly that).

  config1_oracle.json: d = 4 symmetric Gaussian (a = 0.1), 50 bins, 1e5
  samples, 5 iterations, alpha = 1.5, seed 0 -- the per-iteration estimates
  and sigmas (as hex floats), the combination, and a SHA-256 of the final
  grid's FP64 bytes.
  paths_oracle.json: the same records for the other oracle paths on small
  seeded inputs -- a stratified run (d = 3 Genz Gaussian, 2^10 hypercubes of
  4 samples, 3 iterations), one iteration of the LO toy on a 24 x 12 density
  grid, and an observable histogram of a d = 4 Genz Gaussian iteration.
"""
import hashlib
import json
import os
import sys

import numpy as np

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


def _sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a, dtype="<f8").tobytes())
    return h.hexdigest()


def paths():
    from paper_2010_09341_gb300 import workloads as W
    out = {}
    p3 = W.genz_params("genz_gauss", 3, seed=2)
    r = O.integrate_strat(3, 20, "genz_gauss", p3, 10, 4, 3, alpha=1.5, seed=2, integral_id=1)
    out["strat"] = {
        "source": "oracle.integrate_strat(3, 20, 'genz_gauss', genz_params(3, seed=2), B=10, P=4, 3 iterations, seed=2, id=1)",
        "iters": [[float(I).hex(), float(s).hex()] for I, s in r["iters"]],
        "I": float(r["I"]).hex(), "sigma": float(r["sigma"]).hex(),
        "edges_sha256": _sha(r["edges"]),
    }
    xg, u0, u1, v0, v1 = W.pdf_grid(24, 12)
    O.set_pdf_grid(xg, u0, u1, v0, v1)
    acc = O.iterate(3, 20, O.uniform_edges(3, 20), "lo_pdf", W.lo_params(), 0, 0, 0, 20_000)
    out["lo_pdf"] = {
        "source": "oracle.iterate(3, 20, uniform, 'lo_pdf', lo_params(), seed 0, id 0, t 0, 20000) on pdf_grid(24, 12)",
        "S1": float(acc["S1"]).hex(), "S2": float(acc["S2"]).hex(), "hist_sha256": _sha(acc["hist"]),
    }
    p4 = W.genz_params("genz_gauss", 4, seed=3)
    h1, h2 = O.histogram(4, 20, O.uniform_edges(4, 20), "genz_gauss", p4, 3, 8, 0, 20_000, 1, 17, 0.1, 0.9)
    out["histogram"] = {
        "source": "oracle.histogram(4, 20, uniform, 'genz_gauss', genz_params(4, seed=3), seed 3, id 8, t 0, 20000, x_1, 17 bins on [0.1, 0.9))",
        "sha256": _sha(h1, h2),
    }
    return out


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "config1_oracle.json"), "w") as f:
        json.dump(config1(), f, indent=1)
        f.write("\n")
    with open(os.path.join(here, "paths_oracle.json"), "w") as f:
        json.dump(paths(), f, indent=1)
        f.write("\n")
