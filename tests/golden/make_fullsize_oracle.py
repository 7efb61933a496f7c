"""Write tests/golden/fullsize_oracle.json: oracle values at full workload size.

Calls only the CPU FP64 oracle (``oracle/``) on the seeded synthetic
workloads of ``paper_2405_14060_gb300.synth`` (input generators only); the
CUDA path is never run here.  The stored values are the expected results of
the full-size parity tests and the accuracy figures of the benchmark:

* 24x24 grid Ising (576 spins): log Z by bucket elimination along the row
  sweep (Eq. pr), and p(s_v | e) for a seeded subset of spins by
  conditioning, Z(s_v = x) / Z (Eq. mar-prob written out).
* Random 3-regular graph of 200 spins with its 512 evidence sets (10% of the
  spins observed in each): log p(e) for a seeded subset of the sets by
  bucket elimination with the oracle's min-fill order, and for each of them
  p(s_v | e) of a few seeded unobserved spins by conditioning.
* MAP (Eq. log-map) of a 20x20 grid Ising model (400 spins, seed 20240620)
  by max-sum elimination along the row sweep, and of the 300-variable
  Bayesian network with its evidence: the assignment, its log weight and the
  gap to the best assignment that differs from it (oracle.map_gap).

    python tests/golden/make_fullsize_oracle.py [section ...]   # all: ~35 min on 8 cores
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2405_14060_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "fullsize_oracle.json")


def grid24():
    w = synth.workload(2)
    m = w.model
    order = np.arange(m.nvars)                 # row sweep: buckets of width 24
    t0 = time.time()
    lz = oracle.ve_pr(m, order=order)
    spins = sorted(int(v) for v in np.random.default_rng(2).choice(m.nvars, 6, replace=False))
    marg = [oracle.clamped_marginal(m, v, order=order, logz=lz).tolist() for v in spins]
    print(f"grid24: log Z = {lz:.15f}, {len(spins)} spins, {time.time() - t0:.0f} s", flush=True)
    return {"workload": "grid24x24 Ising, seed 20240524", "order": "row sweep",
            "logz": lz, "spins": spins, "marg": marg}


def rrg200_batched():
    w = synth.workload(4)
    m, ev = w.model, w.evid
    rng = np.random.default_rng(4)
    rows = sorted(int(b) for b in rng.choice(ev.shape[0], 8, replace=False))
    out = {"workload": "rrg3-200 Ising, 512 evidence sets (10% observed), seed 20240526",
           "order": "oracle min-fill", "rows": rows, "logz": [], "spins": [], "marg": []}
    t0 = time.time()
    for b in rows:
        lz = oracle.ve_pr(m, ev[b])
        free = np.nonzero(ev[b] < 0)[0]
        spins = sorted(int(v) for v in rng.choice(free, 3, replace=False))
        out["logz"].append(lz)
        out["spins"].append(spins)
        out["marg"].append([oracle.clamped_marginal(m, v, ev[b], logz=lz).tolist()
                            for v in spins])
    print(f"rrg200: {len(rows)} evidence sets, {time.time() - t0:.0f} s", flush=True)
    return out


def grid20_map():
    m = synth.grid_ising(20, 20240620)
    t0 = time.time()
    x, lp, gap = oracle.map_gap(m, order=np.arange(m.nvars))
    print(f"grid20 MAP: log p = {lp:.12f}, gap {gap:.3e}, {time.time() - t0:.0f} s", flush=True)
    return {"workload": "grid20x20 Ising, seed 20240620", "order": "row sweep",
            "assign": [int(v) for v in x], "logp": lp, "gap": gap}


def bn300_map():
    w = synth.workload(3)
    t0 = time.time()
    x, lp, gap = oracle.map_gap(w.model, w.evid[0])
    print(f"bn300 MAP: log p = {lp:.12f}, gap {gap:.3e}, {time.time() - t0:.0f} s", flush=True)
    return {"workload": "300-variable banded Bayesian network, seed 20240525, 20% observed",
            "order": "oracle min-fill", "assign": [int(v) for v in x], "logp": lp, "gap": gap}


SECTIONS = {"grid24": grid24, "rrg200_batched": rrg200_batched, "grid20_map": grid20_map,
            "bn300_map": bn300_map}


def main():
    res = {"note": "written by tests/golden/make_fullsize_oracle.py from the CPU FP64 oracle"}
    if os.path.exists(OUT):
        with open(OUT) as f:
            res.update(json.load(f))
    for name in (sys.argv[1:] or list(SECTIONS)):
        res[name] = SECTIONS[name]()
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
