"""Write the golden fixture tests/golden/l6_seed21.json from the FP64 oracle.

The paper prints no worked example (no spin states, no energies), so the
stored values here are the oracle's, written by this script, which calls
nothing but `oracle/`.  One L = 6 lattice: the oracle's Gaussian couplings
(Philox kind JGEN + Box-Muller) and initial spins (Philox kind INIT) under
seed 21, both rounded once to fp32 so that a GPU run can start from the very
same values.  From that state the fixture records
  * E/N of the initial state (Eq. 1, each bond once);
  * one over-relaxation half-sweep of colour 0 (Sec. 4);
  * one Metropolis half-sweep of colour 1 (Sec. 2; ball proposal, 3 hits,
    T = 0.5), with the oracle's per-site margin of the closest decision;
  * one heat-bath half-sweep of colour 0 (Sec. 2; T = 0.7);
  * two full sweeps of heat-bath (T = 0.7) + 1 over-relaxation, with E/N
    after each.
Floats are written with repr(), so the file holds them exactly.  A change to
the oracle's arithmetic that moves any of them must rewrite the file with
this script (tests/test_oracle_pins.py fails until it does).

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402

L, SEED = 6, 21
PATH = os.path.join(HERE, "l6_seed21.json")


def compute() -> dict:
    """The fixture's content, from the oracle alone."""
    oracle.build()
    J = oracle.gaussian_couplings(L, SEED).astype(np.float32).astype(np.float64)
    s0 = oracle.init_spins(L, SEED).astype(np.float32).astype(np.float64)
    key = oracle.key(SEED)
    out = {"source": "FP64 oracle (oracle/), written by tests/golden/make_golden.py; energy Eq. 1 (each bond "
                     "once), over-relaxation Sec. 4, Metropolis and heat-bath Sec. 2; the paper prints no worked "
                     "example",
           "L": L, "seed": SEED, "J": J.tolist(), "s0": s0.tolist(),
           "energy_s0": oracle.energy(L, J, s0) / L ** 3}

    s = s0.copy()
    oracle.half_sweep(L, J, s, oracle.OR, 0, oracle.Params(key=key, sweep=0))
    out["or_colour0"] = s.tolist()

    s = s0.copy()
    p = oracle.Params(key=key, sweep=3, beta=2.0, step=0.5, hits=3, proposal=oracle.PROP_BALL)
    m = oracle.half_sweep(L, J, s, oracle.MET, 1, p, want_margins=True)
    out["met_colour1"] = {"sweep": 3, "T": 0.5, "hits": 3, "proposal": "ball", "step": 0.5, "spins": s.tolist(),
                          "margins": m.tolist()}

    s = s0.copy()
    oracle.half_sweep(L, J, s, oracle.HB, 0, oracle.Params(key=key, sweep=5, beta=1.0 / 0.7))
    out["hb_colour0"] = {"sweep": 5, "T": 0.7, "spins": s.tolist()}

    s = s0.copy()
    sched = oracle.Schedule(kind=oracle.HB, n_or=1, beta=1.0 / 0.7, energy_every=1)
    n, elog = oracle.sweeps(L, J, s, sched, key, 2)
    out["hb_or_two_sweeps"] = {"T": 0.7, "n_or": 1, "sweeps": n, "spins": s.tolist(), "energy_log": elog.tolist()}
    return out


if __name__ == "__main__":
    data = compute()
    with open(PATH, "w") as f:  # one line per entry
        f.write("{\n" + ",\n".join(f"{json.dumps(k)}: {json.dumps(v)}" for k, v in data.items()) + "\n}\n")
    print(PATH)
