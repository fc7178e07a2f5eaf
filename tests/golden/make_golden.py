"""Write the oracle's per-prefix solution and node counts for the larger boards.

Calls only the CPU oracle (``oracle/``) and the seeded rank generator
(``synth_inputs``): nothing here comes from the CUDA path.

Whole prefix sets, spec ``N:d`` -> ``oracle_n{N}_d{d}.npz``:
  counts  uint64 [num]  solutions below each canonical prefix (unweighted)
  nodes   uint64 [num]  placements in rows d..N-1 below each prefix
  weights uint8  [num]  the prefix weights of the symmetric decomposition
The weighted total is checked against OEIS A000170 before writing.

Seeded samples of a set too large for the oracle, spec ``N:d:k:seed`` ->
``oracle_n{N}_d{d}_s{k}.npz``: k distinct canonical indices drawn uniformly by
SplitMix64 (``synth_inputs.sample_ranks(seed, set size, k)``, in draw order),
with the same three arrays plus
  ranks   uint64 [k]     the canonical indices
  cols    int8   [k, d]  the oracle's own prefix (column of the queen in each row)
No total exists for a sample; the file instead records the set size, which is
checked against the oracle's prefix count.

Usage: python tests/golden/make_golden.py [spec ...]
       (default 16:5 17:5 18:5 19:5 20:7:2048:2020 21:7:2048:2121 22:7:2048:2222)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth_inputs  # noqa: E402

DEFAULT = ["16:5", "17:5", "18:5", "19:5", "20:7:2048:2020", "21:7:2048:2121",
           "22:7:2048:2222"]


def whole(n, d, q):
    t0 = time.time()
    cols, w = oracle.prefixes(n, d)
    counts, nodes = oracle.count_prefixes(n, cols)
    total = sum(int(a) * int(b) for a, b in zip(w, counts))
    if total != q[str(n)]:
        raise SystemExit(f"N={n} d={d}: oracle total {total} != OEIS {q[str(n)]}")
    path = os.path.join(HERE, f"oracle_n{n}_d{d}.npz")
    np.savez_compressed(path, counts=counts, nodes=nodes, weights=w)
    print(f"N={n} d={d}: {len(cols)} prefixes, total {total}, nodes {int(nodes.sum())}, "
          f"{time.time() - t0:.1f}s -> {os.path.basename(path)}", flush=True)


def sample(n, d, k, seed):
    t0 = time.time()
    size = oracle.prefix_count(n, d)
    ranks = np.array(synth_inputs.sample_ranks(seed, size, k), dtype=np.uint64)
    cols = oracle.prefixes_at_ranks(n, d, ranks)
    counts, nodes = oracle.count_prefixes(n, cols)
    # weight of each sampled prefix: 2 except the odd-N centre prefix at d = 1
    # (Section 1's rule as the oracle's own generator applies it)
    wfull = oracle.prefixes(n, d)[1] if d <= 1 else None
    weights = np.array([int(wfull[r]) if wfull is not None else 2 for r in ranks],
                       dtype=np.uint8)
    path = os.path.join(HERE, f"oracle_n{n}_d{d}_s{k}.npz")
    np.savez_compressed(path, ranks=ranks, cols=cols, counts=counts, nodes=nodes,
                        weights=weights, set_size=np.array([size], dtype=np.uint64),
                        seed=np.array([seed], dtype=np.uint64))
    print(f"N={n} d={d}: {k} of {size} prefixes (seed {seed}), solutions "
          f"{int(counts.sum())}, nodes {int(nodes.sum())}, {time.time() - t0:.1f}s -> "
          f"{os.path.basename(path)}", flush=True)


def main(specs):
    q = json.load(open(os.path.join(HERE, "oeis_a000170.json")))["Q"]
    for spec in specs:
        parts = [int(x) for x in spec.split(":")]
        if len(parts) == 2:
            whole(parts[0], parts[1], q)
        elif len(parts) == 4:
            sample(*parts)
        else:
            raise SystemExit(f"bad spec {spec!r}: N:d or N:d:k:seed")


if __name__ == "__main__":
    main(sys.argv[1:] or DEFAULT)
