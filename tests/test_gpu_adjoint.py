"""Hand-written adjoint on the GPU: element-wise against the oracle's
vector-Jacobian product, against central finite differences of the GPU forward
(32^3 binary sub-case), the gravitational-energy identity dE/drho ~ phi dV on the
128^3 binary, and the torch.autograd route."""
import numpy as np
import pytest

import oracle
from paper_2304_11002_gb300 import binding
from paper_2304_11002_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_11002_gb300 import build
    build.build()


def _gpu_vjp(tree, rho, vphi, vg, precision=binding.OCTO_FP64):
    fmm = binding.OctoFMM(tree, 0.5, precision)
    r = torch.from_numpy(np.ascontiguousarray(rho.reshape(-1))).cuda()
    fmm.forces(r)
    dphi = torch.from_numpy(np.ascontiguousarray(vphi)).cuda()
    dg = torch.from_numpy(np.ascontiguousarray(vg)).cuda()
    drho = torch.empty_like(r)
    binding.octo_fmm_backward(fmm.handle, dphi, dg, drho)
    torch.cuda.synchronize()
    binding.octo_fmm_stats(fmm.handle)  # raises if a device-side index check failed
    return drho.cpu().numpy()


@pytest.mark.parametrize("which", ["uniform16", "tiny_adaptive", "unbalanced"])
def test_adjoint_matches_oracle_vjp(which):
    if which == "uniform16":
        w = W.uniform16(5)
        tree, rho = w.tree, w.rho.reshape(-1)
    else:
        refined = {(0, 0, 0, 0), (1, 1, 0, 0)} if which == "tiny_adaptive" else \
            {(0, 0, 0, 0), (1, 0, 0, 0), (2, 1, 1, 1), (3, 3, 3, 3)}
        tree = W.tree_from_refined(refined, 16.0)
        rho = np.random.default_rng(31).lognormal(size=tree.n_leaf * 512)
    n = rho.size
    rng = np.random.default_rng(32)
    vphi, vg = rng.normal(size=n), rng.normal(size=(3, n))
    got = _gpu_vjp(tree, rho, vphi, vg)
    ref = oracle.fmm_vjp(tree, rho, vphi, vg)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= 1e-11, err


def test_adjoint_matches_oracle_vjp_adaptive4():
    """Element by element on the 4-level adaptive binary (interior nodes on three
    levels, refinement boundaries, tabulated and general cross-level pairs)."""
    w = W.adaptive_binary(3, 0.08)
    tree, rho = w.tree, w.rho.reshape(-1)
    n = rho.size
    rng = np.random.default_rng(34)
    vphi, vg = rng.normal(size=n), rng.normal(size=(3, n))
    got = _gpu_vjp(tree, rho, vphi, vg)
    ref = oracle.fmm_vjp(tree, rho, vphi, vg)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= 1e-11, err


@pytest.mark.parametrize("name", ["adaptive4", "adaptive7", "binary128"])
def test_adjoint_dot_product(name):
    """<v, J u> (oracle complex step at 96 sampled cells) against <J^T v, u> (GPU
    adjoint) for v supported on those cells: on the 4-level adaptive binary, on the
    7-level adaptive binary of the benchmark and on the 128^3 differentiation case."""
    w = W.adaptive_binary(3, 0.08) if name == "adaptive4" else W.make(name)
    tree, rho = w.tree, w.rho.reshape(-1)
    n = rho.size
    rng = np.random.default_rng(33)
    idx = np.sort(rng.choice(n, size=96, replace=False))
    mask = np.zeros(n, np.uint8)
    mask[idx] = 1
    vphi = np.zeros(n)
    vg = np.zeros((3, n))
    vphi[idx] = rng.normal(size=idx.size)
    vg[:, idx] = rng.normal(size=(3, idx.size))
    u = rng.normal(size=n) * rho
    _, _, dphi, dg = oracle.fmm_jvp(tree, rho, u, leaf_mask=mask)
    lhs = vphi[idx] @ dphi[idx] + np.sum(vg[:, idx] * dg[:, idx])
    got = _gpu_vjp(tree, rho, vphi, vg)
    assert abs(got @ u - lhs) <= 1e-10 * abs(lhs), (got @ u, lhs)


def test_adjoint_finite_differences_binary32():
    """32^3 sub-case of the 128^3 differentiation config (binary scaled by 1/2):
    loss = sum w g_x with w ~ N(0, 1); central differences of the GPU float64
    forward with h_i = 1e-6 rho_i on 32 cells."""
    w = W.binary32()
    rho = w.rho.reshape(-1).copy()
    n = rho.size
    rng = np.random.default_rng(0)
    wts = rng.normal(size=n)
    vg = np.zeros((3, n))
    vg[0] = wts
    adj = _gpu_vjp(w.tree, rho, np.zeros(n), vg)
    fmm = binding.OctoFMM(w.tree)
    wt = torch.from_numpy(wts).cuda()
    # probe cells inside the stars (where rho is not the floor)
    cand = np.nonzero(rho > 1e-3)[0]
    for i in rng.choice(cand, size=32, replace=False):
        hs = 1e-6 * rho[i]
        vals = []
        for sgn in (1, -1):
            r = rho.copy()
            r[i] += sgn * hs
            _, g = fmm.forces(torch.from_numpy(r).cuda())
            vals.append(float((wt * g[0]).sum()))
        fd = (vals[0] - vals[1]) / (2 * hs)
        assert abs(adj[i] - fd) <= 1e-6 * np.max(np.abs(adj)), (i, adj[i], fd)


def test_energy_gradient_binary128():
    """128^3 binary: E = 1/2 sum rho phi dV, dE/drho = phi dV to expansion accuracy."""
    w = W.binary128()
    rho = w.rho.reshape(-1)
    dV = w.tree.leaf_cell_h() ** 3
    fmm = binding.OctoFMM(w.tree)
    r = torch.from_numpy(rho.copy()).cuda()
    phi, g = fmm.forces(r)
    dphi = (0.5 * r * torch.from_numpy(dV).cuda()).contiguous()
    drho = torch.empty_like(r)
    binding.octo_fmm_backward(fmm.handle, dphi, torch.zeros_like(g), drho)
    torch.cuda.synchronize()
    dE = 0.5 * phi.cpu().numpy() * dV + drho.cpu().numpy()
    ref = phi.cpu().numpy() * dV
    err = np.max(np.abs(dE - ref)) / np.max(np.abs(ref))
    assert err < 1e-3, err


def test_autograd_function():
    from paper_2304_11002_gb300.autograd import fmm_forces
    w = W.uniform16(6)
    fmm = binding.OctoFMM(w.tree)
    rho = torch.from_numpy(w.rho.reshape(-1).copy()).cuda().requires_grad_(True)
    wts = torch.randn(rho.numel(), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    phi, g = fmm_forces(rho, fmm)
    loss = (wts * g[0]).sum() + 0.5 * (phi * rho).sum()
    loss.backward()
    vphi = (0.5 * rho.detach()).cpu().numpy()
    vg = np.zeros((3, rho.numel()))
    vg[0] = wts.cpu().numpy()
    ref = oracle.fmm_vjp(w.tree, w.rho.reshape(-1), vphi, vg) + 0.5 * phi.detach().cpu().numpy()
    got = rho.grad.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
