"""Writes tests/golden/esu_counts.json: exact connected-induced-subgraph counts
of seeded synthetic graphs, by the oracle's ESU enumeration (Wernicke 2006).

Calls only the oracle and the shared input generator.  The generator is
platform independent, so the stored counts hold on any machine.

    python tests/golden/make_goldens.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

GRAPHS = {
    # the 4-node workload: n=2,000, exponent 2.5, mean degree 8, max degree 200, seed 1
    "cl_n2k": dict(gen="workload", name="cl_n2k", ks=(4,)),
    # a small power-law graph for the 1,000-seed statistical tests
    "cl_n200": dict(gen="chung_lu", args=(200, 2.3, 6.0, 30.0), seed=7, ks=(4, 5)),
}


def graph(spec):
    if spec["gen"] == "workload":
        return synth.workload(spec["name"])
    return synth.chung_lu(*spec["args"], seed=spec["seed"])


def main():
    out = {"_source": "exact counts by ESU; written by tests/golden/make_goldens.py"}
    for name, spec in GRAPHS.items():
        rp, col = graph(spec)
        g = oracle.OracleGraph(rp, col)
        entry = {"n": g.n, "nnz": g.nnz, "Gamma": [str(x) for x in g.Gamma],
                 "Lambda3": str(g.Lambda3), "Lambda4": str(g.Lambda4)}
        for k in spec["ks"]:
            entry[f"esu{k}"] = [int(x) for x in g.esu(k)]
        out[name] = entry
        print(name, entry)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "esu_counts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
