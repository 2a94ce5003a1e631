"""The allocation-free entry point mrrr_eigenvalues_static, called through the
C ABI, against the workspace-based solver (mrrr_stein) and the CPU oracle.

mrrr_eigenvalues_static is for callers that cannot call cudaMalloc when they
need eigenvalues (device memory already held by another allocator, or loops
that cannot pay for cudaFree's device-wide synchronisation).  Its scratch is
a static device array shared by all calls, so the test makes two calls in a
row on different matrices -- the second smaller and with a different index
range -- and checks that nothing of the first leaks into the second.  This
file is collected last so that a stop at its first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1205_2107_gb300 import _lib, api, inputs

EPS = 2.0 ** -53


def _dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _static_call(d, e, il, iu, W):
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.mrrr_eigenvalues_static(int(d.numel()), ctypes.c_void_p(d.data_ptr()),
                                       ctypes.c_void_p(e.data_ptr()), il, iu,
                                       ctypes.c_void_p(W.data_ptr()), stream)


@pytest.mark.gpu
def test_two_calls_in_a_row_match_the_workspace_solver():
    cases = [
        inputs.uniform(1500, 1205) + (1, 1500),
        inputs.glued_wilkinson(20) + (5, 300),
        inputs.wilkinson_plus(201) + (150, 201),
    ]
    for d_np, e_np, il, iu in cases:
        n = len(d_np)
        d, e = _dev(d_np), _dev(np.append(e_np, 0.0))
        W = torch.full((iu - il + 1,), -7.0, dtype=torch.float64, device="cuda")
        assert _static_call(d, e, il, iu, W) == _lib.OK
        torch.cuda.synchronize()
        Wref = api.eigh_tridiagonal(d, e, il, iu, vectors=False)
        # the independent checker: the CPU oracle's bisection on T itself
        Wall = oracle.eigvalsh_tridiagonal(d_np, e_np)
        tn = float(np.max(np.abs(Wall)))
        err = float((W - Wref).abs().max())
        assert torch.isfinite(W).all()
        assert bool((W[1:] >= W[:-1]).all()), "W not ascending"
        assert err <= 4 * n * EPS * tn, f"n={n} il={il} iu={iu}: eigenvalue error {err:.3e}"
        err_o = float(np.max(np.abs(W.cpu().numpy() - Wall[il - 1:iu])))
        assert err_o <= 4 * n * EPS * tn, f"n={n} il={il} iu={iu}: error vs oracle {err_o:.3e}"


@pytest.mark.gpu
def test_device_error_gives_nan_and_the_next_call_recovers():
    """A non-finite entry is found on the GPU and gives NaN eigenvalues; the
    next call, on another matrix, rewrites the shared status word and comes
    out right (no state carries over from the failed call)."""
    d_np, e_np = inputs.uniform(700, 77)
    bad = d_np.copy()
    bad[123] = np.nan
    d, e = _dev(bad), _dev(np.append(e_np, 0.0))
    W = torch.zeros(10, dtype=torch.float64, device="cuda")
    assert _static_call(d, e, 1, 10, W) == _lib.OK  # found on the device, not on the host
    torch.cuda.synchronize()
    assert torch.isnan(W).all()
    d2_np, e2_np = inputs.toeplitz(300, 2.0, -1.0)
    d2, e2 = _dev(d2_np), _dev(np.append(e2_np, 0.0))
    W2 = torch.zeros(300, dtype=torch.float64, device="cuda")
    assert _static_call(d2, e2, 1, 300, W2) == _lib.OK
    torch.cuda.synchronize()
    ref = inputs.toeplitz_eigenvalues(300, 2.0, -1.0)
    assert float(np.max(np.abs(W2.cpu().numpy() - ref))) <= 4 * 300 * EPS * 4.0


@pytest.mark.gpu
def test_sizes_beyond_the_maximum_are_rejected():
    n = _lib.STATIC_MAX_N + 1
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    W = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _static_call(d, d, 1, 1, W) == _lib.ERR_ARG
    assert _static_call(d[:10], d[:10], 0, 3, W) == _lib.ERR_ARG
    assert _static_call(d[:0], d[:0], 1, 1, W) == _lib.OK  # n = 0 is a no-op
