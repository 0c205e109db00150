"""Write ``lambda_table.json``: MOSUM critical values for the named workloads.

lambda depends on alpha, the bandwidth h (as a fraction of n) and the horizon
T = N/n, and is found by simulation (Section 2.1, after Eq. 4).  Values here
come from the oracle's Monte-Carlo of the limiting process
W(t) - W(t-h) - h W(1), t in [1, T] (1000 grid steps per unit, 1e5 paths).

Run:  python synth/make_lambda_table.py
"""
import json
import os
import sys

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), ".."))

import oracle  # noqa: E402

G, REPS, SEED = 1000, 100000, 20180704


def main():
    out = {"how": f"oracle.critical_value(alpha, h, T, G={G}, reps={REPS}, seed={SEED})",
           "workloads": {}, "grid_h0.25_alpha0.05": {}}
    specs = {"c1": (0.05, 0.25, 228 / 100), "c2": (0.05, 0.25, 414 / 228), "c3": (0.05, 0.25, 228 / 100)}
    for name, (a, h, T) in specs.items():
        lam = oracle.critical_value(a, h, T, G=G, reps=REPS, seed=SEED)
        out["workloads"][name] = {"alpha": a, "h": h, "T": T, "lambda": round(lam, 4)}
        print(name, T, lam, flush=True)
    for i in range(12, 31):
        T = i / 10
        lam = oracle.critical_value(0.05, 0.25, T, G=G, reps=REPS, seed=SEED)
        out["grid_h0.25_alpha0.05"][f"{T:.1f}"] = round(lam, 4)
        print(T, lam, flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lambda_table.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
