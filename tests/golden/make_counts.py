"""Writes tests/golden/counts_uniform.txt: ordered same-level M2L and P2P counts of
complete octrees (theta = 0.5), taken from the oracle's full dual-tree walk.
Calls only the oracle and the input generators."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2304_11002_gb300 import workloads as W  # noqa: E402

rows = []
for name, lv in [("uniform16", 1), ("binary32", 2), ("binary64", 3), ("binary128", 4)]:
    tree = W.uniform_tree(lv, 8.0 * 2 ** lv)
    c = oracle.counts(tree, 0.5)
    assert c[1] == 0 and c[3] == 0
    rows.append(f"{name} {lv} {c[0]} {c[2]}")
    print(rows[-1], flush=True)
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "counts_uniform.txt"), "w") as f:
    f.write("# name max_level ordered_same_level_M2L ordered_same_level_P2P  (theta 0.5, complete octrees)\n")
    f.write("# written by tests/golden/make_counts.py from the oracle's dual-tree walk\n")
    f.write("\n".join(rows) + "\n")
