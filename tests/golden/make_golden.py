"""Write the oracle's per-prefix solution and node counts for the larger boards.

Calls only the CPU oracle (``oracle/``): nothing here comes from the CUDA path.
For each (N, d) it stores, in ``oracle_n{N}_d{d}.npz``:
  counts  uint64 [num]  solutions below each canonical prefix (unweighted)
  nodes   uint64 [num]  placements in rows d..N-1 below each prefix
  weights uint8  [num]  the prefix weights of the symmetric decomposition
and checks the weighted total against OEIS A000170 before writing.

Usage: python tests/golden/make_golden.py [N:d ...]   (default 16:5 17:5 18:5)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402


def main(specs):
    q = json.load(open(os.path.join(HERE, "oeis_a000170.json")))["Q"]
    for spec in specs:
        n, d = (int(x) for x in spec.split(":"))
        t0 = time.time()
        cols, w = oracle.prefixes(n, d)
        counts, nodes = oracle.count_prefixes(n, cols)
        total = sum(int(a) * int(b) for a, b in zip(w, counts))
        if total != q[str(n)]:
            raise SystemExit(f"N={n} d={d}: oracle total {total} != OEIS {q[str(n)]}")
        path = os.path.join(HERE, f"oracle_n{n}_d{d}.npz")
        np.savez_compressed(path, counts=counts, nodes=nodes, weights=w)
        print(f"N={n} d={d}: {len(cols)} prefixes, total {total}, nodes {int(nodes.sum())}, "
              f"{time.time() - t0:.1f}s -> {os.path.basename(path)}")


if __name__ == "__main__":
    main(sys.argv[1:] or ["16:5", "17:5", "18:5"])
