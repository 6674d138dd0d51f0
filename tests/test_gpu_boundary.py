"""The C ABI's contract beyond the arithmetic: the density check of P2M, the order of
the phase calls that the adjoint relies on, the binding's buffer checks, and the
release of everything create allocated when an allocation fails."""
import os

import numpy as np
import pytest

from paper_2304_11002_gb300 import binding
from paper_2304_11002_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OCTO_ENOMEM, OCTO_ENONPOS, OCTO_ESTATE = -3, -6, -7


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_11002_gb300 import build
    build.build()


@pytest.mark.parametrize("bad", [float("nan"), 0.0, -1.0, float("inf")])
@pytest.mark.parametrize("precision", [binding.OCTO_FP64, binding.OCTO_MIXED])
def test_density_must_be_finite_and_positive(bad, precision):
    w = W.uniform16(0)
    fmm = binding.OctoFMM(w.tree, 0.5, precision)
    rho = w.rho.reshape(-1).copy()
    good = torch.from_numpy(rho.copy()).cuda()
    rho[1234] = bad
    r = torch.from_numpy(rho).cuda()
    fmm.forces(r)  # asynchronous: the check runs on the device
    with pytest.raises(binding.OctoError) as e:
        binding.octo_fmm_stats(fmm.handle)
    assert e.value.code == OCTO_ENONPOS and "finite and positive" in str(e.value)
    # reported once; a valid density afterwards is clean
    fmm.forces(good)
    binding.octo_fmm_stats(fmm.handle)
    # the synchronous host-buffer call reports it directly
    phi_h, g_h = np.empty(rho.size), np.empty((3, rho.size))
    with pytest.raises(binding.OctoError) as e:
        binding.octo_fmm_forces_host(fmm.handle, rho, phi_h, g_h)
    assert e.value.code == OCTO_ENONPOS
    binding.octo_fmm_forces_host(fmm.handle, w.rho.reshape(-1).copy(), phi_h, g_h)
    assert np.all(np.isfinite(phi_h)) and np.all(np.isfinite(g_h))


def test_backward_needs_a_complete_forward():
    w = W.uniform16(1)
    n = w.tree.n_leaf * 512
    fmm = binding.OctoFMM(w.tree)
    r = torch.from_numpy(w.rho.reshape(-1).copy()).cuda()
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((3, n), dtype=torch.float64, device="cuda")
    dphi, dg, drho = torch.ones_like(phi), torch.zeros_like(g), torch.empty_like(phi)

    def backward_code():
        try:
            binding.octo_fmm_backward(fmm.handle, dphi, dg, drho)
            return 0
        except binding.OctoError as e:
            return e.code

    assert backward_code() == OCTO_ESTATE  # nothing ran yet
    binding.octo_fmm_upward(fmm.handle, r)
    binding.octo_fmm_downward(fmm.handle, phi, g)  # interact skipped
    assert backward_code() == OCTO_ESTATE
    binding.octo_fmm_upward(fmm.handle, r)
    binding.octo_fmm_interact(fmm.handle)
    binding.octo_fmm_downward(fmm.handle, phi, g)
    assert backward_code() == 0
    binding.octo_fmm_upward(fmm.handle, 2 * r)  # a new solve has started
    assert backward_code() == OCTO_ESTATE
    binding.octo_fmm_interact(fmm.handle)
    assert backward_code() == OCTO_ESTATE
    binding.octo_fmm_downward(fmm.handle, phi, g)
    assert backward_code() == 0
    fmm.forces(r)
    assert backward_code() == 0
    torch.cuda.synchronize()
    binding.octo_fmm_stats(fmm.handle)


def test_binding_refuses_buffers_the_kernels_would_overrun():
    w = W.uniform16(2)
    n = w.tree.n_leaf * 512
    fmm = binding.OctoFMM(w.tree)
    ok = torch.from_numpy(w.rho.reshape(-1).copy()).cuda()
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((3, n), dtype=torch.float64, device="cuda")
    bad = {
        "float32 rho": (ok.float(), phi, g),
        "short rho": (ok[:-1], phi, g),
        "host rho": (ok.cpu(), phi, g),
        "short phi": (ok, phi[: n - 512], g),
        "short g": (ok, phi, g[:2]),
        "strided g": (ok, phi, torch.empty((n, 3), dtype=torch.float64, device="cuda").t()),
    }
    for what, (r, p, gg) in bad.items():
        with pytest.raises(ValueError):
            binding.octo_fmm_forces(fmm.handle, r, p, gg)
    with pytest.raises(ValueError):
        binding.octo_fmm_backward(fmm.handle, phi, g, phi[:10])
    with pytest.raises(ValueError):
        binding.octo_fmm_forces_host(fmm.handle, np.ones(n - 1), np.empty(n), np.empty((3, n)))
    from paper_2304_11002_gb300.autograd import fmm_forces
    with pytest.raises(ValueError):
        fmm_forces(ok.float().requires_grad_(True), fmm)
    assert binding.octo_fmm_get_option(fmm.handle, 20) == n
    assert binding.octo_fmm_get_option(fmm.handle, 21) == torch.cuda.current_device()
    assert binding.octo_fmm_get_option(fmm.handle, 22) == w.tree.n_nodes


@pytest.mark.parametrize("precision", [binding.OCTO_FP64, binding.OCTO_MIXED])
def test_allocation_failures_release_everything(precision, monkeypatch):
    """Every device allocation of octo_fmm_create failed in turn (test hook): each
    attempt returns OCTO_ENOMEM and leaves the device's free memory as it was."""
    w = W.binary32()
    binding.OctoFMM(w.tree, 0.5, precision)  # loads the kernels and warms the context
    torch.cuda.synchronize()
    base, _ = torch.cuda.mem_get_info()
    failures = 0
    for k in range(1, 200):
        monkeypatch.setenv("OCTO_FMM_FAIL_ALLOC_AT", str(k))
        try:
            h = binding.octo_fmm_create(w.tree, 0.5, 3, precision)
        except binding.OctoError as e:
            assert e.code == OCTO_ENOMEM, (k, str(e))
            failures += 1
            free, _ = torch.cuda.mem_get_info()
            assert free == base, (k, base - free)
            continue
        binding.octo_fmm_destroy(h)  # the k-th allocation did not exist: create succeeded
        break
    else:
        raise AssertionError("create never succeeded")
    monkeypatch.delenv("OCTO_FMM_FAIL_ALLOC_AT")
    assert failures >= 20, failures
    free, _ = torch.cuda.mem_get_info()
    assert free == base
