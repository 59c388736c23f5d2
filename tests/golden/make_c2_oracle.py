"""Write tests/golden/c2_oracle.json: the FP64 oracle's error on the whole
1,000,000-row C2 stream (d = 50,000, l = 100, seed 0; the stream the
benchmark times), computed by the oracle alone.

    python tests/golden/make_c2_oracle.py [--rows N]

Runs Sparse Frequent Directions (Alg. 2 with BoostedSparseShrink, Alg. 4,
and DenseShrink, Alg. 5) in float64 over the stream, then measures
cov-err = ||A^T A - B^T B||_2 / ||A||_F^2 (Sec. 5) and the FD bound
||A - A_k||_F^2 / (l - k) with k = 20. Takes several minutes of CPU time.
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import metrics  # noqa: E402
from oracle import sfd as O  # noqa: E402
from paper_1602_00412_gb300 import synth  # noqa: E402  (seeded input generator only)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", type=int, default=1_000_000)
    ap.add_argument("--out", default=os.path.join(HERE, "c2_oracle.json"))
    a = ap.parse_args()
    d, ell, k, seed = 50000, 100, 20, 0
    X = synth.c2(seed=seed, n=a.rows)
    t0 = time.perf_counter()
    B, o = O.sfd_stream(X.indptr, X.indices, X.values, d, ell, seed)
    t_sketch = time.perf_counter() - t0
    A = X.to_scipy()
    fro2 = metrics.fro2(A)
    cov = metrics.cov_norm_psd(A, B)
    tail = metrics.tail_mass(A, k)
    out = {
        "workload": "c2: planted(n=%d, d=50000, Poisson(50), Zipf(1.1), rank 20, 10*0.8^t, "
                    "noise 0.1), seed 0" % a.rows,
        "rows": int(X.n), "nnz": int(X.nnz), "d": d, "ell": ell, "k": k, "seed": seed,
        "buffers": len(o.log), "attempts": int(sum(e["attempts"] for e in o.log)),
        "q": sorted({int(e["q"]) for e in o.log if e["q"] is not None}),
        "fro2": fro2, "cov_norm": cov, "cov_err": cov / fro2,
        "tail_mass": tail, "fd_bound": tail / (ell - k),
        "oracle_seconds": round(t_sketch, 1),
        "made_by": "tests/golden/make_c2_oracle.py (oracle/ only)",
    }
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
