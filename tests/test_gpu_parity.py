"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by
element, on the same seeded inputs (float64 path: relative tolerance 1e-12)."""
import numpy as np
import pytest

import oracle
from paper_2304_11002_gb300 import binding
from paper_2304_11002_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _rel_phi(phi, ref, idx=None):
    if idx is not None:
        phi, ref = phi[idx], ref[idx]
    return float(np.max(np.abs(phi - ref) / np.abs(ref)))


def _rel_g(g, ref, idx=None):
    if idx is not None:
        g, ref = g[:, idx], ref[:, idx]
    return float(np.max(np.linalg.norm(g - ref, axis=0)) / np.max(np.linalg.norm(ref, axis=0)))


def _run(tree, rho, precision=binding.OCTO_FP64, theta=0.5, graph=True):
    fmm = binding.OctoFMM(tree, theta, precision)
    if not graph:
        binding.octo_fmm_set_option(fmm.handle, 1, 0)
    r = torch.from_numpy(np.ascontiguousarray(rho.reshape(-1))).cuda()
    phi, g = fmm.forces(r)
    torch.cuda.synchronize()
    binding.octo_fmm_stats(fmm.handle)  # raises on a device-side error (e.g. a bounded wait that ran out)
    return fmm, phi.cpu().numpy(), g.cpu().numpy()


def _tiny_adaptive():
    return W.tree_from_refined({(0, 0, 0, 0), (1, 1, 0, 0)}, 16.0)


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_11002_gb300 import build
    build.build()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_uniform16_fp64_full(seed):
    w = W.uniform16(seed)
    fmm, phi, g = _run(w.tree, w.rho)
    po, go, _ = oracle.fmm(w.tree, w.rho)
    assert _rel_phi(phi, po) <= TOL64
    assert _rel_g(g, go) <= TOL64


def test_uniform16_multipoles_and_locals():
    w = W.uniform16(0)
    fmm, phi, g = _run(w.tree, w.rho)
    mp = binding.octo_fmm_read_state(fmm.handle, 0, w.tree.n_nodes)
    mo = oracle.upward(w.tree, w.rho)
    for f in range(20):
        s = np.max(np.abs(mo[f])) or 1.0
        assert np.max(np.abs(mp[f] - mo[f])) <= TOL64 * s, f
    loc = binding.octo_fmm_read_state(fmm.handle, 1, w.tree.n_nodes)
    _, _, lo = oracle.fmm(w.tree, w.rho, want_local=True)
    interior = np.repeat(~w.tree.is_leaf, 512)
    for f in range(23):
        a, b = loc[f][interior], lo[f][interior]
        s = np.max(np.abs(b)) or 1.0
        assert np.max(np.abs(a - b)) <= TOL64 * s, f


def test_tiny_adaptive_fp64_full():
    tree = _tiny_adaptive()
    rho = np.random.default_rng(11).lognormal(size=(tree.n_leaf, 512))
    fmm, phi, g = _run(tree, rho)
    po, go, _ = oracle.fmm(tree, rho)
    assert _rel_phi(phi, po) <= TOL64
    assert _rel_g(g, go) <= TOL64


def _unbalanced():
    """A tree that is not 2:1 balanced: level-3 subgrids next to level-1 leaves, so
    cross-level pairs two levels apart (general cross-level kernel) occur beside the
    tabulated one-level pairs."""
    return W.tree_from_refined({(0, 0, 0, 0), (1, 0, 0, 0), (2, 1, 1, 1), (3, 3, 3, 3)}, 16.0)


def _stage_names(fmm):
    return [binding.octo_fmm_stage_info(fmm.handle, i)["name"] for i in range(binding.octo_fmm_stage_count(fmm.handle))]


@pytest.mark.parametrize("precision", [binding.OCTO_FP64, binding.OCTO_MIXED])
def test_unbalanced_tree_full(precision):
    tree = _unbalanced()
    rho = np.random.default_rng(12).lognormal(size=(tree.n_leaf, 512))
    fmm, phi, g = _run(tree, rho, precision)
    names = _stage_names(fmm)
    # tabulated one-level pairs: their own stage (per-kind launches) or cross items of
    # the persistent queue whose sums a short stage applies afterwards
    assert any(n in ("cross_cells", "cross_cells_apply") for n in names) and "cross_leaf" in names, names
    po, go, _ = oracle.fmm(tree, rho)
    tol = TOL64 if precision == binding.OCTO_FP64 else 1e-6
    assert _rel_phi(phi, po) <= tol
    assert _rel_g(g, go) <= tol


def _sample(n_cells, k, seed):
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(n_cells, size=min(k, n_cells), replace=False))
    mask = np.zeros(n_cells, dtype=np.uint8)
    mask[idx] = 1
    return idx, mask


@pytest.mark.parametrize("name", ["adaptive4", "binary64", "adaptive7", (1000, 0.3, 1), (1000, 1.0, 2), "star5"])
def test_sampled_cells_fp64(name):
    """Full-size trees (64^3 uniform binary; 7-level adaptive binary with ~8000
    leaf subgrids; throughput-sweep trees of ~1000 leaf subgrids with mass ratios
    0.3 and 1 and rotated axes): every cell computed on the GPU, a seeded sample of
    cells by the oracle."""
    if isinstance(name, tuple):
        w = W.sweep(name[0], q=name[1], seed=name[2])
    else:
        w = W.adaptive_binary(3, 0.08) if name == "adaptive4" else W.make(name)
    fmm, phi, g = _run(w.tree, w.rho)
    idx, mask = _sample(w.tree.n_leaf * 512, 192, 5)
    po, go, _ = oracle.fmm(w.tree, w.rho, leaf_mask=mask)
    assert _rel_phi(phi, po, idx) <= TOL64
    assert _rel_g(g, go, idx) <= TOL64
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(g))


def test_counts_from_handle_match_oracle():
    tree = W.adaptive_binary(3, 0.08).tree
    fmm = binding.OctoFMM(tree)
    np.testing.assert_array_equal(fmm.counts(), oracle.counts(tree))


def test_homogeneity_and_determinism_bit_exact():
    w = W.adaptive_binary(3, 0.08)
    fmm = binding.OctoFMM(w.tree)
    r = torch.from_numpy(w.rho.reshape(-1).copy()).cuda()
    phi1, g1 = [x.clone() for x in fmm.forces(r)]
    phi2, g2 = [x.clone() for x in fmm.forces(r)]
    phi3, g3 = [x.clone() for x in fmm.forces(2 * r)]
    assert torch.equal(phi1, phi2) and torch.equal(g1, g2)
    assert torch.equal(phi3, 2 * phi1) and torch.equal(g3, 2 * g1)


def test_graph_and_phases_and_host_path_agree():
    w = W.adaptive_binary(3, 0.08)
    fmm = binding.OctoFMM(w.tree)
    r = torch.from_numpy(w.rho.reshape(-1).copy()).cuda()
    phi1, g1 = [x.clone() for x in fmm.forces(r)]
    phi2 = torch.empty_like(phi1)
    g2 = torch.empty_like(g1)
    binding.octo_fmm_upward(fmm.handle, r)
    binding.octo_fmm_interact(fmm.handle)
    binding.octo_fmm_downward(fmm.handle, phi2, g2)
    torch.cuda.synchronize()
    assert torch.equal(phi1, phi2) and torch.equal(g1, g2)
    rho_h = w.rho.reshape(-1).copy()
    phi_h = np.empty_like(rho_h)
    g_h = np.empty((3, rho_h.size))
    binding.octo_fmm_forces_host(fmm.handle, rho_h, phi_h, g_h)
    assert np.array_equal(phi_h, phi1.cpu().numpy()) and np.array_equal(g_h, g1.cpu().numpy())


def test_conservation_on_gpu_output():
    """Newton III and angular momentum (Section IV-C) hold for the GPU forces."""
    tree = _tiny_adaptive()
    rho = np.random.default_rng(12).lognormal(size=(tree.n_leaf, 512))
    _, phi, g = _run(tree, rho)
    m = rho.reshape(-1) * tree.leaf_cell_h() ** 3
    x = tree.leaf_cell_centres()
    F = (m[None, :] * g).T
    assert np.linalg.norm(F.sum(0)) <= 1e-13 * np.abs(F).sum()
    tau = np.cross(x, F)
    assert np.linalg.norm(tau.sum(0)) <= 1e-13 * np.abs(tau).sum()


def test_errors_are_reported():
    w = W.uniform16(0)
    with pytest.raises(binding.OctoError) as e:
        binding.octo_fmm_create(w.tree, 0.5, 4, binding.OCTO_FP64)
    assert e.value.code == -1
    fmm = binding.OctoFMM(w.tree)
    d = torch.empty(4096, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.OctoError) as e:
        binding.octo_fmm_backward(fmm.handle, d, torch.empty((3, 4096), dtype=torch.float64, device="cuda"), d)
    assert e.value.code == -7


@pytest.mark.parametrize("precision", [binding.OCTO_FP64, binding.OCTO_MIXED])
def test_interaction_strategies_bit_identical(precision):
    """Per-kind launches and the persistent work queue (every register budget, merged
    or paced) run the same item functions: identical results for every interior shape (mixed
    precision: 32 or 64 stencil entries per float32 partial sum, half- or
    quarter-node items), each shape within the mixed tolerance of the oracle, and
    the autotuner picks one of the candidates."""
    w = W.adaptive_binary(3, 0.08)
    r = torch.from_numpy(w.rho.reshape(-1).copy()).cuda()
    mixed = precision == binding.OCTO_MIXED
    budgets = (1, 2, 3) if mixed else (1, 2)
    shapes = [(32, 1), (64, 1), (32, 2), (64, 2)] if mixed else [None]
    po, go, _ = oracle.fmm(w.tree, w.rho) if mixed else (None, None, None)
    cross = None
    first = None
    # schedules: per-kind launches, the merged persistent queue under every register
    # budget and (mixed precision) the paced persistent queue
    schedules = [(1, 1, 0)] + [(2, b, 0) for b in budgets] + ([(2, 3, 1), (2, 1, 1)] if mixed else [])
    for shape in shapes:
        outs = []
        for mode, minb, paced in schedules:
            fmm = binding.OctoFMM(w.tree, 0.5, precision)
            binding.octo_fmm_set_option(fmm.handle, 3, mode)
            binding.octo_fmm_set_option(fmm.handle, 4, minb)
            if shape is not None:
                binding.octo_fmm_set_option(fmm.handle, 6, shape[0])
                binding.octo_fmm_set_option(fmm.handle, 7, shape[1])
                binding.octo_fmm_set_option(fmm.handle, 8, paced)
            phi, g = fmm.forces(r)
            outs.append((phi.clone(), g.clone()))
            names = _stage_names(fmm)
            if mode == 1:
                cross = "cross_cells" in names
            else:  # the tabulated cross-level pairs ran as items of the persistent queue
                assert ("cross_cells_apply" in names) == cross, names
        assert cross  # this tree has tabulated cross-level pairs
        for phi, g in outs[1:]:
            assert torch.equal(phi, outs[0][0]) and torch.equal(g, outs[0][1]), shape
        if mixed:
            p, gg = outs[0][0].cpu().numpy(), outs[0][1].cpu().numpy()
            assert _rel_phi(p, po) <= 1e-6 and _rel_g(gg, go) <= 1e-6, shape
        if first is None:
            first = outs[0]
    fmm = binding.OctoFMM(w.tree, 0.5, precision)
    phi, g = fmm.forces(r)
    assert binding.octo_fmm_get_option(fmm.handle, 3) in (1, 2)
    assert all(binding.octo_fmm_get_option(fmm.handle, k) > 0 for k in [10 + b for b in (0,) + budgets])
    if precision == binding.OCTO_FP64:
        assert binding.octo_fmm_get_option(fmm.handle, 13) == 0
        with pytest.raises(binding.OctoError):
            binding.octo_fmm_set_option(fmm.handle, 4, 3)
        assert torch.equal(phi, first[0]) and torch.equal(g, first[1])
    else:
        shape = (binding.octo_fmm_get_option(fmm.handle, 6), binding.octo_fmm_get_option(fmm.handle, 7))
        assert shape in shapes
        assert binding.octo_fmm_get_option(fmm.handle, 14) > 0 and binding.octo_fmm_get_option(fmm.handle, 15) > 0
        if binding.octo_fmm_get_option(fmm.handle, 3) == 2:  # the paced queue was timed
            assert binding.octo_fmm_get_option(fmm.handle, 16) > 0
        assert _rel_phi(phi.cpu().numpy(), po) <= 1e-6 and _rel_g(g.cpu().numpy(), go) <= 1e-6
