"""The autograd wrappers' marshalling, on the CPU.

The library calls (api.eigh_tridiagonal, api.eigh_tridiagonal_batched,
api.eigh_tridiagonal_backward) are replaced by CPU stand-ins with the same
packing conventions: dense eigh for the solve, the oracle's dense gradient
formula for the backward pass.  What is tested is the wrappers' own work:
transposes between (n, k) views and column-major storage, packing of W, Z and
the gradients, the trailing entry of e, padded inputs, n = 0 and n = 1, and
the recompute path.  The GPU kernels themselves are tested in
test_gpu_backward.py."""
import numpy as np
import pytest
import torch

import oracle
from paper_1205_2107_gb300 import api, autograd

F64 = torch.float64


def _eig(d, e):
    n = len(d)
    if n == 0:
        return np.zeros(0), np.zeros((0, 0))
    W, V = np.linalg.eigh(oracle.tridiag_dense(d, e[:n - 1]))
    return W, V


def fake_single(d, e, il=None, iu=None, *, vectors=True, plan=None, check=True):
    W, V = _eig(d.numpy(), e.numpy())
    Zt = torch.tensor(V.T.copy(), dtype=F64)  # contiguous (k, n): row j = column j of Z
    return torch.tensor(W, dtype=F64), Zt.t()


def fake_batched(d, e, layout, *, vectors=True, plan=None, check=True, out=None):
    W = torch.zeros(max(layout.k_total, 1), dtype=F64)
    Z = torch.zeros(max(layout.z_total, 1), dtype=F64)
    dn, en = d.numpy(), e.numpy()
    for p, n in enumerate(layout.sizes):
        r0, w0, z0 = layout.offsets_host[p], layout.w_offsets_host[p], layout.z_offsets_host[p]
        Wp, V = _eig(dn[r0:r0 + n], en[r0:r0 + n])
        W[w0:w0 + n] = torch.tensor(Wp)
        Z[z0:z0 + n * n] = torch.tensor(V.T.reshape(-1).copy())  # column-major block
    return W, Z


def fake_backward(W, Z, Wbar, Zbar, layout, *, tau_rel=0.0, plan=None, check=True):
    dbar = torch.zeros(max(layout.n_total, 1), dtype=F64)
    ebar = torch.zeros(max(layout.n_total, 1), dtype=F64)
    for p, n in enumerate(layout.sizes):
        if n == 0:
            continue
        r0, w0, z0 = layout.offsets_host[p], layout.w_offsets_host[p], layout.z_offsets_host[p]
        Wp = W[w0:w0 + n].numpy()
        Zp = Z[z0:z0 + n * n].numpy().reshape(n, n).T  # column j = eigenvector j
        Wb = Wbar[w0:w0 + n].numpy() if Wbar is not None else None
        Zb = Zbar[z0:z0 + n * n].numpy().reshape(n, n).T if Zbar is not None else None
        tau = tau_rel * float(np.max(np.abs(Wp)))
        gd, ge = oracle.adjoint(Wp, Zp, Wb, Zb, tau=tau)
        dbar[r0:r0 + n] = torch.tensor(gd)
        ebar[r0:r0 + n - 1] = torch.tensor(ge)
    return dbar, ebar


@pytest.fixture
def cpu_library(monkeypatch):
    monkeypatch.setattr(api, "eigh_tridiagonal", fake_single)
    monkeypatch.setattr(api, "eigh_tridiagonal_batched", fake_batched)
    monkeypatch.setattr(api, "eigh_tridiagonal_backward", fake_backward)


def loss_np(d, e, w, C):
    """Sign-invariant loss sum w_i lambda_i + sum (c_i^T z_i)^2 by dense eigh."""
    W, V = _eig(d, e)
    return float(w @ W + np.sum(np.einsum("ji,ji->i", C, V) ** 2))


def fd_grad(d, e, w, C, h=1e-6):
    gd, ge = np.zeros_like(d), np.zeros(max(len(d) - 1, 0))
    for j in range(len(d)):
        dp, dm = d.copy(), d.copy()
        dp[j] += h
        dm[j] -= h
        gd[j] = (loss_np(dp, e, w, C) - loss_np(dm, e, w, C)) / (2 * h)
    for j in range(len(d) - 1):
        ep, em = e.copy(), e.copy()
        ep[j] += h
        em[j] -= h
        ge[j] = (loss_np(d, ep, w, C) - loss_np(d, em, w, C)) / (2 * h)
    return gd, ge


@pytest.mark.parametrize("e_len", ["n-1", "n"])
@pytest.mark.parametrize("recompute", [False, True])
def test_single_problem_gradient(cpu_library, e_len, recompute):
    rng = np.random.default_rng(4)
    n = 9
    d_np, e_np = rng.standard_normal(n), rng.standard_normal(n - 1)
    w_np, C_np = rng.standard_normal(n), rng.standard_normal((n, n))
    e_in = e_np if e_len == "n-1" else np.append(e_np, 7.0)
    d = torch.tensor(d_np, requires_grad=True)
    e = torch.tensor(e_in, requires_grad=True)
    W, Z = autograd.eigh_tridiagonal_autograd(d, e, recompute=recompute)
    loss = (torch.tensor(w_np) * W).sum() + ((torch.tensor(C_np) * Z).sum(0) ** 2).sum()
    loss.backward()
    gd, ge = fd_grad(d_np, e_np, w_np, C_np)
    assert d.grad.shape == d.shape and e.grad.shape == e.shape
    assert np.allclose(d.grad.numpy(), gd, atol=1e-6, rtol=1e-6)
    assert np.allclose(e.grad.numpy()[:n - 1], ge, atol=1e-6, rtol=1e-6)
    if e_len == "n":
        assert e.grad[-1].item() == 0.0


def test_single_problem_edge_sizes(cpu_library):
    for n in (0, 1):
        d = torch.ones(n, dtype=F64, requires_grad=True)
        e = torch.zeros(max(n - 1, 0), dtype=F64, requires_grad=True)
        W, Z = autograd.eigh_tridiagonal_autograd(d, e)
        (3.0 * W.sum() + Z.sum() * 0.0).backward()
        assert d.grad.shape == (n,)
        assert torch.equal(d.grad, torch.full((n,), 3.0, dtype=F64))


def test_batched_gradient_matches_single_and_padding_gets_zero(cpu_library):
    rng = np.random.default_rng(8)
    sizes = [3, 0, 6, 1]
    lay = api.BatchLayout(sizes, "cpu")
    ds = [rng.standard_normal(n) for n in sizes]
    es = [np.append(rng.standard_normal(max(n - 1, 0)), 0.0)[:n] for n in sizes]
    ws = [rng.standard_normal(n) for n in sizes]
    Cs = [rng.standard_normal((n, n)) for n in sizes]
    pad = 2  # packed inputs longer than n_total
    d = torch.tensor(np.concatenate(ds + [np.full(pad, 5.0)]), requires_grad=True)
    e = torch.tensor(np.concatenate(es + [np.full(pad, 5.0)]), requires_grad=True)
    W, Z = autograd.eigh_tridiagonal_batched_autograd(d, e, lay)
    loss = 0.0
    for p, n in enumerate(sizes):
        w0, z0 = lay.w_offsets_host[p], lay.z_offsets_host[p]
        Zp = Z[z0:z0 + n * n].view(n, n).t()  # column-major block -> (n, n), column j = z_j
        loss = loss + (torch.tensor(ws[p]) * W[w0:w0 + n]).sum() + ((torch.tensor(Cs[p]) * Zp).sum(0) ** 2).sum()
    loss.backward()
    assert d.grad.shape == d.shape and e.grad.shape == e.shape
    assert torch.all(d.grad[-pad:] == 0) and torch.all(e.grad[-pad:] == 0)
    for p, n in enumerate(sizes):
        if n == 0:
            continue
        r0 = lay.offsets_host[p]
        gd, ge = fd_grad(ds[p], es[p], ws[p], Cs[p])
        assert np.allclose(d.grad[r0:r0 + n].numpy(), gd, atol=1e-6, rtol=1e-6)
        assert np.allclose(e.grad[r0:r0 + n - 1].numpy(), ge, atol=1e-6, rtol=1e-6)
        assert e.grad[r0 + n - 1].item() == 0.0


def test_batched_autograd_refuses_subsets(cpu_library):
    lay = api.BatchLayout([4], "cpu", il=[1], iu=[2])
    with pytest.raises(ValueError, match="all eigenpairs"):
        autograd.eigh_tridiagonal_batched_autograd(torch.zeros(4, dtype=F64, requires_grad=True),
                                                   torch.zeros(4, dtype=F64), lay)
