"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/octo_fmm.h declares, and its host-side planner agrees with the oracle's
tree walk on the interaction counts and rejects malformed trees."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2304_11002_gb300 import binding, build
from paper_2304_11002_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(octo_fmm_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    L = binding.lib()
    declared = _declared_symbols()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared == set(binding.SYMBOLS)


def _tiny_adaptive():
    return W.tree_from_refined({(0, 0, 0, 0), (1, 1, 0, 0)}, 16.0)


@pytest.mark.parametrize("which", ["uniform16", "binary32", "tiny_adaptive", "adaptive4"])
def test_plan_counts_match_oracle_walk(which):
    if which == "uniform16":
        tree = W.uniform16(0).tree
    elif which == "binary32":
        tree = W.binary32().tree
    elif which == "tiny_adaptive":
        tree = _tiny_adaptive()
    else:
        tree = W.adaptive_binary(3, 0.08).tree
    c_lib = binding.octo_fmm_plan_counts(tree, 0.5)
    c_orc = oracle.counts(tree, 0.5)
    np.testing.assert_array_equal(c_lib, c_orc)


def test_plan_rejects_bad_trees():
    tree = W.uniform16(0).tree
    bad = W.Tree(tree.level.copy(), tree.ijk.copy(), tree.children.copy(), tree.origin, tree.extent)
    bad.children[0, 3] = -1  # 7 children
    with pytest.raises(binding.OctoError) as e:
        binding.octo_fmm_plan_counts(bad)
    assert e.value.code == -2
    bad = W.Tree(tree.level.copy(), tree.ijk.copy(), tree.children.copy(), tree.origin, tree.extent)
    bad.ijk[1] = [1, 1, 1]  # child at the wrong octant
    with pytest.raises(binding.OctoError) as e:
        binding.octo_fmm_plan_counts(bad)
    assert e.value.code == -2
    with pytest.raises(binding.OctoError) as e:
        binding.octo_fmm_plan_counts(tree, theta=0.3)  # near field beyond the 26 neighbours
    assert e.value.code == -1
