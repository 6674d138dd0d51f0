"""The allocation-free entry point (octo_fmm_subgrids_noalloc) through the C ABI,
against the allocating path (octo_fmm_create + octo_fmm_forces on a one-node tree)
within the float64 tolerance of the other parity tests, on two calls in a row.
It is meant for callers that cannot allocate device memory when they call the
solver (under a memory manager that owns all device memory, or in a loop that
must not stall on an allocation).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2304_11002_gb300 import binding
from paper_2304_11002_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_11002_gb300 import build
    build.build()


def _reference(rho_sub, h):
    """phi, g of one 8^3 subgrid through the allocating entry points."""
    tree = W.tree_from_refined(set(), 8.0 * h)
    fmm = binding.OctoFMM(tree, 0.5, binding.OCTO_FP64)
    phi, g = fmm.forces(torch.from_numpy(np.ascontiguousarray(rho_sub)).cuda())
    torch.cuda.synchronize()
    return phi.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("calls", [((5, 0.25, 1), (3, 2.0, 2))])
def test_noalloc_matches_allocating_path_twice(calls):
    for n, h, seed in calls:
        rho = np.random.default_rng(seed).lognormal(size=n * 512)
        r = torch.from_numpy(rho).cuda()
        phi = torch.empty(n * 512, dtype=torch.float64, device="cuda")
        g = torch.empty((3, n * 512), dtype=torch.float64, device="cuda")
        binding.octo_fmm_subgrids_noalloc(n, r, h, phi, g)
        torch.cuda.synchronize()
        phi, g = phi.cpu().numpy(), g.cpu().numpy()
        for s in range(n):
            po, go = _reference(rho[s * 512:(s + 1) * 512], h)
            sl = slice(s * 512, (s + 1) * 512)
            assert np.max(np.abs(phi[sl] - po) / np.abs(po)) <= TOL64
            assert np.max(np.linalg.norm(g[:, sl] - go, axis=0)) <= TOL64 * np.max(np.linalg.norm(go, axis=0))


def test_noalloc_rejects_oversize_batch():
    n = 1025 * 512
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((3, n), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.OctoError) as e:
        binding.octo_fmm_subgrids_noalloc(1025, d, 1.0, d, g)
    assert e.value.code == -1 and "1024" in str(e.value)


def _raw(n, rho, h, phi, g):
    """The C symbol itself (no binding-side checks), on the current stream."""
    L = binding.lib()
    p = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    rc = L.octo_fmm_subgrids_noalloc(int(n), p(rho), float(h), p(phi), p(g),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    msg = L.octo_fmm_last_error(None)
    return rc, (msg.decode() if msg else "")


@pytest.mark.parametrize("case", ["n=-1", "h=0", "h=-1", "h=nan", "rho=null", "phi=null", "g=null"])
def test_noalloc_rejects_bad_arguments(case):
    d = torch.zeros(512, dtype=torch.float64, device="cuda")
    g = torch.zeros((3, 512), dtype=torch.float64, device="cuda")
    n, h, rho, phi, gg = 1, 1.0, d, d.clone(), g
    if case == "n=-1":
        n = -1
    elif case.startswith("h="):
        h = {"h=0": 0.0, "h=-1": -1.0, "h=nan": float("nan")}[case]
    elif case == "rho=null":
        rho = None
    elif case == "phi=null":
        phi = None
    else:
        gg = None
    rc, msg = _raw(n, rho, h, phi, gg)
    assert rc == -1
    want = {"n": "n_subgrids", "h": "cell width", "r": "null buffer", "p": "null buffer", "g": "null buffer"}[case[0]]
    assert want in msg, msg


def test_noalloc_empty_batch_is_a_no_op():
    phi = torch.full((512,), 7.0, dtype=torch.float64, device="cuda")
    rc, _ = _raw(0, phi, 1.0, phi, torch.zeros((3, 512), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert rc == 0 and bool(torch.all(phi == 7.0))


def test_noalloc_second_call_allocates_nothing():
    """The first call on a device loads the module (which is when the driver
    reserves the fixed array); from then on a call changes no device memory."""
    n = 4
    rho = torch.from_numpy(np.random.default_rng(3).lognormal(size=n * 512)).cuda()
    phi = torch.empty(n * 512, dtype=torch.float64, device="cuda")
    g = torch.empty((3, n * 512), dtype=torch.float64, device="cuda")
    binding.octo_fmm_subgrids_noalloc(n, rho, 0.5, phi, g)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        binding.octo_fmm_subgrids_noalloc(n, rho, 0.5, phi, g)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
