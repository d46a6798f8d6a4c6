"""The allocation-free residual-norm entry point agrees with the library's own residual.

Some callers cannot allocate device memory (for example while another allocator
holds all free HBM, or when an allocation's implicit device synchronisation is
not acceptable).  ddamg_residual_norm_noalloc serves them: it computes
||b - D x|| / ||b|| with a fixed file-scope scratch array instead of a
cudaMalloc'ed buffer.  This test checks it, through the C ABI, against the true
residual that ddamg_solve reports for the same (b, x), twice in a row (the
scratch array is shared and reused between calls).  It lives in its own file,
collected last, and builds its own hierarchy so it also runs alone.
"""
import numpy as np
import pytest

import synth
from cases import Case, SMALL2

pytestmark = pytest.mark.gpu


def test_residual_norm_noalloc_matches_solve_twice():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    import paper_1307_6101_gb300 as dd
    c = Case(**SMALL2, max_rhs=3, n_inv=1, eta_passes=2, m0=-0.3)
    h = c.gpu(1)
    b = torch.from_numpy(np.ascontiguousarray(synth.random_spinors(3, c.dims, 11))).cuda()
    x = torch.zeros_like(b)
    stats = dd.ddamg_solve(h, b, x, 3, 1e-10)
    ref = np.array([s["true_residual"] for s in stats])
    # At a solution b - D x is pure cancellation: an FP64 application of D agrees to
    # 1e-12 relative to ||D x|| ~ ||b||, hence an absolute 1e-12 on ||b - D x|| / ||b||.
    for _ in range(2):
        out_host = np.zeros(3)
        dd.ddamg_residual_norm_noalloc(h, b, x, 3, out_host)
        assert np.allclose(out_host, ref, rtol=1e-12, atol=1e-12), (out_host, ref)
        out_dev = torch.zeros(3, dtype=torch.float64, device="cuda")
        dd.ddamg_residual_norm_noalloc(h, b, x, 3, out_dev)
        assert np.allclose(out_dev.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)
    # a non-solution (O(1) residual) against the residual computed from ddamg_apply
    y = torch.from_numpy(np.ascontiguousarray(synth.random_spinors(3, c.dims, 12))).cuda()
    Dy = torch.zeros_like(y)
    dd.ddamg_apply(h, 0, 0, y, Dy, 3)
    expect = np.linalg.norm((b - Dy).cpu().numpy().reshape(3, -1), axis=1) / np.linalg.norm(
        b.cpu().numpy().reshape(3, -1), axis=1)
    out_host = np.zeros(3)
    dd.ddamg_residual_norm_noalloc(h, b, y, 3, out_host)
    assert np.allclose(out_host, expect, rtol=1e-12, atol=0)
    with pytest.raises(dd.DdamgError):
        dd.ddamg_residual_norm_noalloc(h, b, x, 65, out_host)
