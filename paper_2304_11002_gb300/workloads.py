"""Seeded synthetic inputs: octrees of 8^3-cell subgrids and density fields.

This module holds no FMM arithmetic.  It builds the tree descriptor (level, ijk,
children arrays, the same plain arrays the C-ABI takes) and samples densities at
leaf-cell centres.  Both the CUDA path's tests and the oracle's tests take their
inputs from here.

Node order: level by level, Morton order of ijk within a level.  Leaf order (the
layout of rho, phi and g) is the node order restricted to leaves; inside a leaf
the 512 cells are x-fastest: local = a + 8 b + 64 c.

Workload recipes (the paper's v1309 / DWD inputs are not available, so these
stand in for them, following its binary-star scenarios of Section IV-C):
  uniform16   16^3 cells, 2 levels, lognormal(0, 1) density per cell
  binary64    64^3 cells, 4 levels, two n=1.5 polytropes (R 12 and 10 cells, mass
              ratio 0.7, separation 30 cells) + 1e-10 floor
  adaptive7   7 levels (0..6), refinement where rho > 1e-4 rho_max on a binary
              (q = 0.7, n = 1.5), 2:1 balanced, about 8000 leaf subgrids
  binary128   128^3 cells, 5 levels, binary64 scaled by 2
  sweep       adaptive trees of about 1e3 / 1e4 / 5e4 leaf subgrids
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, Optional, Tuple

import numpy as np

FLOOR = 1e-10


@dataclasses.dataclass
class Tree:
    level: np.ndarray      # int32 [n]
    ijk: np.ndarray        # int32 [n, 3]
    children: np.ndarray   # int32 [n, 8], -1 for leaves; octant o = ox + 2 oy + 4 oz
    origin: np.ndarray     # float64 [3]
    extent: float

    @property
    def n_nodes(self) -> int:
        return int(self.level.shape[0])

    @property
    def is_leaf(self) -> np.ndarray:
        return self.children[:, 0] < 0

    @property
    def leaf_nodes(self) -> np.ndarray:
        return np.nonzero(self.is_leaf)[0].astype(np.int32)

    @property
    def n_leaf(self) -> int:
        return int(self.is_leaf.sum())

    @property
    def max_level(self) -> int:
        return int(self.level.max())

    def h(self, level: int) -> float:
        return self.extent / (8.0 * 2.0 ** level)

    def leaf_cell_centres(self) -> np.ndarray:
        """[n_leaf*512, 3] geometric centres of leaf cells in leaf order."""
        a = np.arange(512)
        loc = np.stack([a & 7, (a >> 3) & 7, a >> 6], axis=1).astype(np.float64)
        out = []
        for nd in self.leaf_nodes:
            h = self.h(int(self.level[nd]))
            out.append(self.origin + h * (8.0 * self.ijk[nd] + loc + 0.5))
        return np.concatenate(out, axis=0) if out else np.zeros((0, 3))

    def leaf_cell_h(self) -> np.ndarray:
        """[n_leaf*512] cell width of every leaf cell."""
        return np.repeat([self.h(int(self.level[nd])) for nd in self.leaf_nodes], 512)


def _morton(i: int, j: int, k: int) -> int:
    code = 0
    for b in range(21):
        code |= ((i >> b) & 1) << (3 * b) | ((j >> b) & 1) << (3 * b + 1) | ((k >> b) & 1) << (3 * b + 2)
    return code


def tree_from_refined(refined: set, extent: float, origin=(0.0, 0.0, 0.0)) -> Tree:
    """Tree whose interior nodes are exactly `refined` ((level, i, j, k) tuples)."""
    levels = [[(0, 0, 0, 0)]]
    while True:
        nxt = []
        for (l, i, j, k) in levels[-1]:
            if (l, i, j, k) in refined:
                for o in range(8):
                    nxt.append((l + 1, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1), 2 * k + ((o >> 2) & 1)))
        if not nxt:
            break
        nxt.sort(key=lambda t: _morton(t[1], t[2], t[3]))
        levels.append(nxt)
    nodes = [t for lv in levels for t in lv]
    index = {t: n for n, t in enumerate(nodes)}
    n = len(nodes)
    level = np.array([t[0] for t in nodes], dtype=np.int32)
    ijk = np.array([t[1:] for t in nodes], dtype=np.int32).reshape(n, 3)
    children = np.full((n, 8), -1, dtype=np.int32)
    for t, idx in index.items():
        if t in refined:
            l, i, j, k = t
            for o in range(8):
                children[idx, o] = index[(l + 1, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1), 2 * k + ((o >> 2) & 1))]
    return Tree(level, ijk, children, np.asarray(origin, dtype=np.float64), float(extent))


def uniform_tree(max_level: int, extent: float) -> Tree:
    refined = set()
    for l in range(max_level):
        s = 1 << l
        for i in range(s):
            for j in range(s):
                for k in range(s):
                    refined.add((l, i, j, k))
    return tree_from_refined(refined, extent)


def balance_2to1(refined: set) -> set:
    """Close `refined` so that leaf nodes sharing a face, edge or corner differ by
    at most one level: every same-level neighbour of a refined node must exist."""
    refined = set(refined)
    changed = True
    while changed:
        changed = False
        for (l, i, j, k) in list(refined):
            if l == 0:
                continue
            s = 1 << l
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    for dk in (-1, 0, 1):
                        a, b, c = i + di, j + dj, k + dk
                        if not (0 <= a < s and 0 <= b < s and 0 <= c < s):
                            continue
                        p = (l - 1, a >> 1, b >> 1, c >> 1)
                        if p not in refined:
                            refined.add(p)
                            changed = True
    # parents of refined nodes must be refined too
    for (l, i, j, k) in list(refined):
        while l > 0:
            l, i, j, k = l - 1, i >> 1, j >> 1, k >> 1
            refined.add((l, i, j, k))
    return refined


def adaptive_tree(box_refine: Callable[[int, np.ndarray, np.ndarray], bool], max_level: int, extent: float,
                  balance: bool = True) -> Tree:
    """Refine node (level l, box [lo, hi)) while box_refine(l, lo, hi) and l < max_level."""
    refined = set()
    frontier = [(0, 0, 0, 0)]
    while frontier:
        nxt = []
        for (l, i, j, k) in frontier:
            if l >= max_level:
                continue
            w = extent / (1 << l)
            lo = np.array([i, j, k], dtype=np.float64) * w
            if box_refine(l, lo, lo + w):
                refined.add((l, i, j, k))
                for o in range(8):
                    nxt.append((l + 1, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1), 2 * k + ((o >> 2) & 1)))
        frontier = nxt
    if balance:
        refined = balance_2to1(refined)
    return tree_from_refined(refined, extent)


# ---------------------------------------------------------------------------
# Density fields
# ---------------------------------------------------------------------------

def lane_emden(n: float = 1.5, dxi: float = 1e-4) -> Tuple[np.ndarray, np.ndarray]:
    """theta_n(xi) by classic RK4 from the series start xi0 = dxi, up to the first zero.
    Returns (xi, theta) samples; xi[-1] is the first zero xi_1 (linear interpolation)."""
    xi = dxi
    th = 1.0 - xi * xi / 6.0 + n * xi ** 4 / 120.0
    dth = -xi / 3.0 + n * xi ** 3 / 30.0

    def f(x, y, dy):
        return dy, -(max(y, 0.0) ** n) - 2.0 * dy / x

    xs, ths = [0.0, xi], [1.0, th]
    while th > 0:
        k1 = f(xi, th, dth)
        k2 = f(xi + dxi / 2, th + dxi / 2 * k1[0], dth + dxi / 2 * k1[1])
        k3 = f(xi + dxi / 2, th + dxi / 2 * k2[0], dth + dxi / 2 * k2[1])
        k4 = f(xi + dxi, th + dxi * k3[0], dth + dxi * k3[1])
        th_new = th + dxi / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        dth_new = dth + dxi / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        if th_new <= 0:
            xi1 = xi + dxi * th / (th - th_new)
            xs.append(xi1)
            ths.append(0.0)
            break
        xi, th, dth = xi + dxi, th_new, dth_new
        xs.append(xi)
        ths.append(th)
    return np.array(xs), np.array(ths)


_LE_CACHE: Dict[float, Tuple[np.ndarray, np.ndarray]] = {}


def polytrope_profile(n: float = 1.5):
    if n not in _LE_CACHE:
        _LE_CACHE[n] = lane_emden(n)
    return _LE_CACHE[n]


def polytrope_density(x: np.ndarray, centre, radius: float, rho_c: float, n: float = 1.5) -> np.ndarray:
    """rho_c theta_n(xi_1 r / R)^n inside r < R, 0 outside."""
    xs, ths = polytrope_profile(n)
    xi1 = xs[-1]
    r = np.linalg.norm(x - np.asarray(centre), axis=1)
    xi = xi1 * r / radius
    th = np.interp(xi, xs, ths, right=0.0)
    out = rho_c * np.maximum(th, 0.0) ** n
    out[r >= radius] = 0.0
    return out


def polytrope_threshold_radius(radius: float, rho_c: float, rho_thr: float, n: float = 1.5) -> float:
    """Radius where rho_c theta^n falls to rho_thr (radius if never)."""
    xs, ths = polytrope_profile(n)
    if rho_thr >= rho_c:
        return 0.0
    t = (rho_thr / rho_c) ** (1.0 / n)
    # theta decreases monotonically on [0, xi_1]
    idx = np.searchsorted(-ths, -t)
    idx = min(max(idx, 1), len(xs) - 1)
    x0, x1, t0, t1 = xs[idx - 1], xs[idx], ths[idx - 1], ths[idx]
    xi = x0 + (t0 - t) * (x1 - x0) / (t0 - t1) if t0 != t1 else x0
    return radius * xi / xs[-1]


@dataclasses.dataclass
class Binary:
    c1: np.ndarray
    c2: np.ndarray
    r1: float
    r2: float
    rho_c1: float
    rho_c2: float
    n: float = 1.5

    def density(self, x: np.ndarray) -> np.ndarray:
        return (polytrope_density(x, self.c1, self.r1, self.rho_c1, self.n)
                + polytrope_density(x, self.c2, self.r2, self.rho_c2, self.n) + FLOOR)


def make_binary(c1, c2, r1, r2, q, sample_points: np.ndarray, cell_volume: np.ndarray, n: float = 1.5) -> Binary:
    """Binary with rho_c1 = 1 and rho_c2 set so that the discrete masses on the given
    sample points have ratio M2 / M1 = q."""
    c1 = np.asarray(c1, dtype=np.float64)
    c2 = np.asarray(c2, dtype=np.float64)
    m1 = float(np.sum(polytrope_density(sample_points, c1, r1, 1.0, n) * cell_volume))
    m2 = float(np.sum(polytrope_density(sample_points, c2, r2, 1.0, n) * cell_volume))
    return Binary(c1, c2, r1, r2, 1.0, q * m1 / m2, n)


# ---------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    tree: Tree
    rho: np.ndarray  # float64 [n_leaf, 512]
    theta: float = 0.5
    note: str = ""


def uniform16(seed: int = 0) -> Workload:
    tree = uniform_tree(1, 16.0)
    rng = np.random.default_rng(seed)
    rho = rng.lognormal(mean=0.0, sigma=1.0, size=(tree.n_leaf, 512))
    return Workload("uniform16", tree, rho, 0.5, f"16^3 lognormal(0,1) seed {seed}")


def _uniform_binary(max_level: int, scale: float, q: float = 0.7) -> Workload:
    extent = 8.0 * 2 ** max_level
    tree = uniform_tree(max_level, extent)
    x = tree.leaf_cell_centres()
    vol = tree.leaf_cell_h() ** 3
    mid = extent / 2.0 + 0.5
    sep = 30.0 * scale
    b = make_binary((mid - sep / 2, mid, mid), (mid + sep / 2, mid, mid), 12.0 * scale, 10.0 * scale, q, x, vol)
    rho = b.density(x).reshape(tree.n_leaf, 512)
    return Workload(f"binary{int(extent)}", tree, rho, 0.5,
                    f"{int(extent)}^3 uniform, n=1.5 binary R={12*scale:g},{10*scale:g} sep={sep:g} q={q}")


def binary64() -> Workload:
    return _uniform_binary(3, 1.0)


def binary128() -> Workload:
    return _uniform_binary(4, 2.0)


def binary32() -> Workload:
    return _uniform_binary(2, 0.5)


def adaptive_binary(max_level: int, r1_frac: float, q: float = 0.7, seed: int = 0, extent: float = 1.0,
                    name: Optional[str] = None) -> Workload:
    """Binary of n=1.5 polytropes in a cubic domain; R2 = (10/12) R1, separation
    2.5 R1.  The seed rotates the binary axis in the x-y plane by a uniform angle and
    shifts the pair by a uniform offset below one finest cell.  Nodes are refined
    where their box meets a cell with rho > 1e-4 rho_max, then 2:1 balanced."""
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0.0, 2.0 * math.pi) if seed else 0.0
    hf = extent / (8.0 * 2 ** max_level)
    shift = rng.uniform(0.0, hf, size=3) if seed else np.zeros(3)
    r1 = r1_frac * extent
    r2 = r1 * 10.0 / 12.0
    sep = 2.5 * r1
    mid = np.full(3, extent / 2.0) + shift
    axis = np.array([math.cos(ang), math.sin(ang), 0.0])
    c1 = mid - axis * sep * 0.5
    c2 = mid + axis * sep * 0.5
    # central densities from continuum masses (rho_c1 = 1): M ~ rho_c R^3 for equal n
    rho_c2 = q * (r1 / r2) ** 3
    rho_max = max(1.0, rho_c2)
    t1 = polytrope_threshold_radius(r1, 1.0, 1e-4 * rho_max)
    t2 = polytrope_threshold_radius(r2, rho_c2, 1e-4 * rho_max)

    def box_refine(l, lo, hi):
        for c, t in ((c1, t1), (c2, t2)):
            p = np.clip(c, lo, hi)
            if np.sum((p - c) ** 2) < t * t:
                return True
        return False

    tree = adaptive_tree(box_refine, max_level, extent)
    x = tree.leaf_cell_centres()
    vol = tree.leaf_cell_h() ** 3
    b = make_binary(c1, c2, r1, r2, q, x, vol)
    rho = b.density(x).reshape(tree.n_leaf, 512)
    nm = name or f"adaptive{max_level + 1}_q{q}_s{seed}"
    return Workload(nm, tree, rho, 0.5,
                    f"adaptive {max_level + 1} levels, R1={r1_frac:g} L, q={q}, seed {seed}, {tree.n_leaf} leaf subgrids")


def adaptive7(seed: int = 0) -> Workload:
    """7 levels (0..6), about 8000 leaf subgrids."""
    return adaptive_binary(6, 0.125, 0.7, seed, name="adaptive7")


def rotating_star(max_level: int, r_frac: float, seed: int = 0, extent: float = 1.0,
                  name: Optional[str] = None) -> Workload:
    """One n=1.5 polytrope of radius r_frac * extent at the domain centre (the rotating
    star of the paper's distributed runs; rotation does not enter the gravity solve).
    The seed shifts the star by a uniform offset below one finest cell.  Nodes are
    refined where their box meets the rho > 1e-4 rho_c region, then 2:1 balanced;
    the density has a 1e-10 floor outside the star."""
    rng = np.random.default_rng(seed)
    hf = extent / (8.0 * 2 ** max_level)
    shift = rng.uniform(0.0, hf, size=3) if seed else np.zeros(3)
    c = np.full(3, extent / 2.0) + shift
    r = r_frac * extent
    t = polytrope_threshold_radius(r, 1.0, 1e-4)

    def box_refine(l, lo, hi):
        p = np.clip(c, lo, hi)
        return bool(np.sum((p - c) ** 2) < t * t)

    tree = adaptive_tree(box_refine, max_level, extent)
    x = tree.leaf_cell_centres()
    rho = (polytrope_density(x, c, r, 1.0) + 1e-10).reshape(tree.n_leaf, 512)
    nm = name or f"star{max_level}_s{seed}"
    return Workload(nm, tree, rho, 0.5,
                    f"rotating star, max level {max_level}, R={r_frac:g} L, seed {seed}, {tree.n_leaf} leaf subgrids")


# max level -> star radius / L close to the paper's rotating-star sizes (5048, 27840
# and 172208 subgrids at levels 5, 6, 7); seed 0 gives 5160, 27784, 169968 leaf subgrids
STAR = {
    5: 0.262,
    6: 0.256,
    7: 0.25,
}


def star(level: int, seed: int = 0) -> Workload:
    return rotating_star(level, STAR[level], seed, name=f"star{level}")


SWEEP = {  # target leaf subgrids -> (max level, R1 / L); q = 0.7, seed 0 gives 960 / 9976 / 50268
    1000: (5, 0.075),
    10000: (6, 0.137),
    50000: (7, 0.133),
}


def sweep(target: int, q: float = 0.7, seed: int = 0) -> Workload:
    ml, r1 = SWEEP[target]
    return adaptive_binary(ml, r1, q, seed, name=f"sweep{target}_q{q}_s{seed}")


RECIPES = {
    "uniform16": uniform16,
    "binary32": binary32,
    "binary64": binary64,
    "binary128": binary128,
    "adaptive7": adaptive7,
}


def make(name: str, **kw) -> Workload:
    if name.startswith("sweep"):
        return sweep(int(name[5:]), **kw)
    if name.startswith("star"):
        return star(int(name[4:]), **kw)
    return RECIPES[name](**kw)


def scf_binary(name: str = "binary32"):
    """Initial guess and surface cells of an SCF run on one of the uniform binaries:
    (workload, params) with params as octo_scf_params takes them (n = 1.5; each star
    keeps the maximum density of its initial polytrope; surface cells A, B = the
    cells nearest to the outer and inner edge of star 1 on the line through both
    centres, C = nearest to the inner edge of star 2; x_split = midway between the
    inner edges)."""
    scale = {"binary32": 0.5, "binary64": 1.0, "binary128": 2.0}[name]
    w = {"binary32": binary32, "binary64": binary64, "binary128": binary128}[name]()
    extent = float(w.tree.extent)
    mid = extent / 2.0 + 0.5
    sep, r1, r2 = 30.0 * scale, 12.0 * scale, 10.0 * scale
    c1, c2 = mid - sep / 2, mid + sep / 2
    x = w.tree.leaf_cell_centres()

    def nearest(px):
        return int(np.argmin(np.linalg.norm(x - np.array([px, mid, mid]), axis=1)))

    rho = w.rho.reshape(-1)
    split = 0.5 * ((c1 + r1) + (c2 - r2))
    star1 = x[:, 0] < split
    params = {"n": 1.5, "rho_max": (float(rho[star1].max()), float(rho[~star1].max())), "rho_floor": 1e-10,
              "cell_a": nearest(c1 - r1), "cell_b": nearest(c1 + r1), "cell_c": nearest(c2 - r2),
              "x_split": split}
    return w, params
