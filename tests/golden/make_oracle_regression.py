"""Write oracle_regression.json: fingerprints of short oracle runs, one per
model and path (Ising 2D/3D and spin-S, North-East, Potts, couplings and
fields, the random-site algorithm and its balanced variant, Phi overlaps).

These are regression fixtures, not pins: they come from the oracle itself
and only guard it against unnoticed changes (the pins that tie it to the
paper and to exact results are the tests/test_oracle_*.py files).  Run
from the repository root:  python tests/golden/make_oracle_regression.py
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

OUT = os.path.join(HERE, "oracle_regression.json")


def _signs(n, seed):
    return np.where(np.random.default_rng(seed).random(n) < 0.5, -1, 1).astype(np.int8)


def cases():
    """name -> (constructor kwargs, extra set-up, run) for each fixture."""
    return {
        "ising2d_L16_T2.27": dict(dims=2, L=16, two_S=1, model=oracle.ISING, J=1.0, h=0.0, T=2.269185, seed=1),
        "ising2d_L12_field": dict(dims=2, L=12, two_S=1, model=oracle.ISING, J=1.0, h=0.3, T=2.0, seed=2),
        "ising3d_L6_spin1": dict(dims=3, L=6, two_S=2, model=oracle.ISING, J=1.0, h=0.0, T=3.0, seed=3),
        "ising2d_L8_spin3/2": dict(dims=2, L=8, two_S=3, model=oracle.ISING, J=1.0, h=-0.2, T=4.0, seed=4),
        "ne_L16_c0.3": dict(dims=2, L=16, two_S=1, model=oracle.NE, J=0.0, h=0.0, T=0.3, seed=5,
                            init=oracle.INIT_EQUILIBRIUM),
        "potts_q3_L12": dict(dims=2, L=12, two_S=2, model=oracle.POTTS, J=1.0, h=0.1, T=1.0, seed=6),
        "spin_glass_fields_L12": dict(dims=2, L=12, two_S=1, model=oracle.ISING, J=1.0, h=0.5, T=1.5, seed=7,
                                      bonds=True, fields=True),
        "rsite_ne_L16_b8_l4": dict(dims=2, L=16, two_S=1, model=oracle.NE, J=0.0, h=0.0, T=0.42, seed=8,
                                   init=oracle.INIT_EQUILIBRIUM, rsite=(8, 4, False)),
        "rsite_balanced_ising_L16_b8_l2": dict(dims=2, L=16, two_S=1, model=oracle.ISING, J=1.0, h=0.0, T=2.3,
                                              seed=9, rsite=(8, 2, True)),
    }


def fingerprint(c, n=12):
    o = oracle.Lattice(c["dims"], c["L"], c["two_S"], c["model"], c["J"], c["h"], c["T"], seed=c["seed"],
                       init=c.get("init", oracle.INIT_RANDOM))
    N = c["L"] ** c["dims"]
    if c.get("bonds"):
        o.set_couplings(_signs(c["dims"] * N, c["seed"] + 100))
    if c.get("fields"):
        o.set_fields(_signs(N, c["seed"] + 200))
    o.set_reference()
    if "rsite" in c:
        b, lam, bal = c["rsite"]
        ser = o.rsite_sweep(n, b, lam, balanced=bal)
    else:
        ser = o.sweep(n)
    out = {"spins_sha256": hashlib.sha256(o.spins.tobytes()).hexdigest()}
    for k in ("bond", "mag", "up", "unflipped", "overlap", "field"):
        if k in ser:
            out[k] = [int(v) for v in ser[k]]
    return out


def main():
    data = {name: fingerprint(c) for name, c in cases().items()}
    with open(OUT, "w") as f:   # one fixture per line
        f.write("{\n")
        names = sorted(data)
        for i, name in enumerate(names):
            f.write("%s: %s%s\n" % (json.dumps(name), json.dumps(data[name], sort_keys=True),
                                    "," if i + 1 < len(names) else ""))
        f.write("}\n")
    print("wrote", OUT, len(data), "fixtures")


if __name__ == "__main__":
    main()
