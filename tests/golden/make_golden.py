"""Writes the oracle regression fixtures of tests/golden/.

Calls only the CPU oracle (and the seeded input generator).  The paper
prints no worked example, so these fixtures pin the oracle to its own
earlier output: a change to its arithmetic shows up here and must be
justified by the passage of the paper (or the stated reading) it follows.

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

CASES = {
    "lattice17_small_grid": dict(k=2, grid_scale=0.01, n=48, precision=0),
    "lattice17_small_grid_fp32": dict(k=2, grid_scale=0.01, n=48, precision=1),
    "infinite_medium_4nuc": dict(k=1, grid_scale=1.0, n=48, precision=0),
}


def case_lines(name):
    c = CASES[name]
    p = synth.make_config(c["k"], n_particles=c["n"], grid_scale=c["grid_scale"])
    r = oracle.run(p, seed=p.seed, batch=3, n=c["n"], threads=1, precision=c["precision"])
    lines = [f"# {name}: config {c['k']} grid_scale {c['grid_scale']} batch 3 precision {c['precision']}",
             "# id n_coll status n_flights n_draws E x y z"]
    for k in range(c["n"]):
        lines.append(" ".join([str(k), str(int(r["n_coll"][k])), str(int(r["status"][k])),
                               str(int(r["n_flights"][k])), str(int(r["n_draws"][k])),
                               float(r["E"][k]).hex(), float(r["x"][k]).hex(),
                               float(r["y"][k]).hex(), float(r["z"][k]).hex()]))
    return lines


if __name__ == "__main__":
    for name in CASES:
        with open(os.path.join(HERE, name + ".txt"), "w") as f:
            f.write("\n".join(case_lines(name)) + "\n")
        print("wrote", name)
