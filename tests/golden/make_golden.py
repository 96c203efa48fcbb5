"""Writes the oracle fixtures in this folder.  Calls only oracle/ and the seeded
input generators; run it from the repository root:  python tests/golden/make_golden.py

The paper prints no worked kernel values (its parity plots, Fig. kernelmatrix_compare,
are images), so these fixtures freeze the pinned oracle's output for the
16-point n=8 reps=2 workload (features iid uniform on [0, pi), seed 0) and a few
reps=1..3 pairs, computed by both oracle constructions.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle  # noqa: E402
from paper_2405_02630_gb300.inputs import workload, uniform_features  # noqa: E402


def main():
    out = {}
    X, _, n, reps = workload("cfg0_n8_r2_N16")
    K_sv = oracle.sv_gram(X, reps)
    K_mps, LK = oracle.mps_gram(X, reps)
    assert np.max(np.abs(K_sv - K_mps)) < 1e-12
    out["cfg0_n8_r2_N16"] = {"source": "oracle O1 state vector (gate by gate), cross-checked against O2 to 1e-12",
                             "n_qubits": n, "reps": reps, "seed": 0, "X": X.tolist(), "K": K_sv.tolist()}
    pairs = []
    for reps in (1, 2, 3):
        Xp = uniform_features(6, 10, 50 + reps)
        for a in range(0, 6, 2):
            k, amp = oracle.sv_kernel_pair(Xp[a], Xp[a + 1], reps)
            pairs.append({"reps": reps, "xi": Xp[a].tolist(), "xj": Xp[a + 1].tolist(), "K": k})
    out["pairs_n10"] = {"source": "oracle O1 state vector, Algorithm 1 recipe per pair", "pairs": pairs}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_fixtures.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
