"""Write tests/golden/c3_first_buffer.json: the FP64 oracle's
BoostedSparseShrink (Alg. 4 over Alg. 3 and Alg. 1, VerifySpectral of
Alg. 6) of the first buffer of the chunk-parallel C3 stream, computed by the
oracle alone.

    python tests/golden/make_c3_oracle.py

The buffer is the first 200,000 rows of chunk 0 (the buffer closes at rows =
d = 200,000: its ~18.4M entries stay below l d = 40M); chunk 0 is sketched
with seed 0, so its first buffer draws the Philox keys (seed 0, b 0, r).
Takes a few minutes of CPU time.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import sfd as O  # noqa: E402
from paper_1602_00412_gb300 import synth  # noqa: E402  (seeded input generator only)


def main():
    d, ell, seed, b = 200000, 200, 0, 0
    X = synth.c3_chunk(seed, 0).rows(0, d)
    A = X.to_scipy()
    q = O.q_fixed(X.n)
    t0 = time.perf_counter()
    Bp, info = O.boosted_sparse_shrink(A, ell, 0.01, seed, b, q)
    lam2 = np.sort(np.asarray(info["lam"]) ** 2)[::-1]
    out = {
        "workload": "c3_chunk(seed 0, chunk 0), rows 0..200000 (first buffer), d = 200000, l = 200",
        "rows": int(X.n), "nnz": int(X.nnz), "d": d, "ell": ell, "seed": seed, "b": b, "q": q,
        "attempts": int(info["attempts"]), "verified": bool(info["verified"]),
        "vs_steps": int(info["p"]), "logsum": info["logsum"], "delta": info["Delta"],
        "fro2_a": float(A.multiply(A).sum()), "fro2_b": float((Bp * Bp).sum()),
        "captured": float(lam2.sum()), "lam2_top": [float(x) for x in lam2[:10]],
        "lam2_ell": float(lam2[ell - 1]),
        "oracle_seconds": round(time.perf_counter() - t0, 1),
        "made_by": "tests/golden/make_c3_oracle.py (oracle/ only)",
    }
    with open(os.path.join(HERE, "c3_first_buffer.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
