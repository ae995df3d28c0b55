"""Writes tests/golden/oracle_small_worlds.json: the FP64 oracle's results on two small seeded
worlds, a regression record of the oracle's arithmetic (the paper prints no worked example).

Only oracle/ and the seeded input generator are called. Run from the repository root:
    python tests/golden/make_golden.py
A change to these values must come with a change to the oracle whose commit names the passage
(or the reading of it) that justifies it.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import coral_oracle as O          # noqa: E402
from paper_2406_09654_gb300 import worlds      # noqa: E402

# (name, world arguments, first step, steps): a one-layer direct-net world across the
# day/night boundary, and a CPPN world with rotation, radiation and merges.
CASES = [
    ("direct_8x6", dict(width=8, height=6, n_genomes=3, hidden=0, net="direct", seed=3,
                        random_rotation=True), 98, 4),
    ("cppn_radiation_10x7", dict(width=10, height=7, n_genomes=4, hidden=16, net="cppn", seed=5,
                                 random_rotation=True, radiation_every=2, p_mut=0.05, p_merge=0.05,
                                 capacity=16), 0, 4),
]


def oracle_case(kw, t0, steps):
    w = worlds.make_world(**kw)
    st = O.State.from_world(w)
    p = O.Params.from_world(w)
    gen = None
    if w.genes is not None:
        gen = O.Genomes.from_genes(w.genes, w.capacity)
        nets = O.nets_from_genomes(gen, w.hidden)
    else:
        nets = O.Nets.from_dense(w.dense, w.hidden, w.capacity)
    tot = []

    def on_step(t, s, info):
        d = O.totals(s)
        tot.append({"t": t, "E": d["E"], "I": d["I"], "C": [float(c) for c in d["C"]],
                    "n_explore": int(info["n_explore"]), "n_takeover": int(info["n_takeover"])})

    st, nets, gen, _ = O.run(st, nets, gen, t0, steps, p, on_step=on_step)
    out = {"totals": tot,
           "E": [float(v) for v in st.E.ravel()], "I": [float(v) for v in st.I.ravel()],
           "G": [int(v) for v in st.G.ravel()], "R": [int(v) for v in st.R.ravel()]}
    if gen is not None:
        out["parent"] = [int(v) for v in gen.parent]
    return out


def build():
    return {name: {"world": kw, "t0": t0, "steps": steps, "oracle": oracle_case(kw, t0, steps)}
            for name, kw, t0, steps in CASES}


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small_worlds.json")
    with open(path, "w") as f:
        json.dump(build(), f, indent=1)
    print(path)
