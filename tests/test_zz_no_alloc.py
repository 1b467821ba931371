"""The allocation-free reduction entry point, called through the C ABI.

lbm_reduce_field_noalloc serves callers that cannot allocate device memory
(their host application owns the device pool, or they may not call
cudaMalloc/cudaFree). It must give the same statistics as lbm_reduce, which
uses a solver workspace, on consecutive calls that reuse its fixed scratch.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from paper_1603_09577_gb300 import Solver
from paper_1603_09577_gb300 import _lib as C

pytestmark = pytest.mark.gpu


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def close(a, b):
    """The FP64 bar of the parity tests (1e-12 relative), exact for counts and maxima."""
    for j in range(8):
        if j in (5, 6):
            assert a[j] == b[j], (j, a[j], b[j])
        else:
            assert abs(a[j] - b[j]) <= 1e-12 * max(abs(b[j]), 1e-300), (j, a[j], b[j])


def test_noalloc_matches_workspace_reduction_twice():
    L = C.lib()
    nx, ny = 301, 257                      # 77,357 values: ten blocks of the scratch, ragged tail
    phi0 = W.phi0_aniso(nx, seed=11, ny=ny)
    s = Solver(nx, ny, prec="f64", bc=("abb", "periodic"), phi_wall=(0.2, 0.4, 0.0, 0.0))
    s.set_coeffs(conv=1, u=(0.06, -0.04), diff=2, K=(0.02, 0.008, 0.01), s=W.s9(), r1=-0.1)
    s.set_phi(torch.from_numpy(phi0).cuda())
    ref = torch.from_numpy(np.random.default_rng(12).uniform(0, 1, (ny, nx))).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        s.step(7)
        phi = s.phi(torch.float64)
        expected = s.reduce_async(ref).cpu().tolist()
        got = torch.full((8,), -1.0, dtype=torch.float64, device="cuda")
        C.check(L.lbm_reduce_field_noalloc(ptr(phi), ptr(ref), phi.numel(), ptr(got), stream))
        close(got.cpu().tolist(), expected)
        # without a reference field the error sums are zero
        got2 = torch.full((8,), -1.0, dtype=torch.float64, device="cuda")
        C.check(L.lbm_reduce_field_noalloc(ptr(phi), None, phi.numel(), ptr(got2), stream))
        g2 = got2.cpu().tolist()
        assert g2[1] == g2[2] == g2[3] == g2[4] == 0.0
        close([g2[0], 0, 0, 0, 0, g2[5], g2[6], g2[7]], [expected[0], 0, 0, 0, 0, expected[5], expected[6], expected[7]])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = C.lib()
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    phi = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = L.lbm_reduce_field_noalloc(ptr(phi), None, 67108864 + 1, ptr(out), None)
    assert rc == C.LBM_EINVAL and b"scratch capacity" in L.lbm_last_error()
    assert L.lbm_reduce_field_noalloc(ptr(phi), None, 0, ptr(out), None) == C.LBM_EINVAL
    assert L.lbm_reduce_field_noalloc(None, None, 16, ptr(out), None) == C.LBM_EINVAL


@pytest.mark.parametrize("n", [4096 * 4096, 67108864])
def test_noalloc_large_fields_fill_the_scratch(n):
    """16,777,216 values (2,048 scratch slots, so the second pass walks more
    partials than it has threads) and exactly the 67,108,864-value capacity (every
    slot): the statistics equal their numpy FP64 definitions, and a second call
    over the reused scratch returns the same bits."""
    L = C.lib()
    g = torch.Generator(device="cuda").manual_seed(n % 1000)
    phi = torch.rand(n, generator=g, dtype=torch.float64, device="cuda") - 0.25
    ref = torch.rand(n, generator=g, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for _ in range(2):
        got = torch.full((8,), -1.0, dtype=torch.float64, device="cuda")
        C.check(L.lbm_reduce_field_noalloc(ptr(phi), ptr(ref), n, ptr(got), stream))
        outs.append(got.cpu())
    assert torch.equal(outs[0], outs[1])
    a, r = phi.cpu().numpy(), ref.cpu().numpy()
    d = a - r
    expected = [a.sum(), np.abs(d).sum(), np.abs(r).sum(), (d * d).sum(), (r * r).sum(), np.abs(a).max(), 0.0,
                (a * a).sum()]
    got = outs[0].tolist()
    for j in range(8):
        if j in (5, 6):
            assert got[j] == expected[j], (j, got[j], expected[j])
        else:
            assert abs(got[j] - expected[j]) <= 1e-12 * abs(expected[j]), (j, got[j], expected[j])
