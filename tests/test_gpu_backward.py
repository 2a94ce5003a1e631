"""GPU parity of the backward pass (mrrr_backward and the autograd wrappers)
against the oracle's dense reference gradient, computed from the oracle's
own eigendecomposition, and against central finite differences of the loss
sum_i w_i lambda_i + sum_i (c_i^T z_i)^2 (w, C iid normal from a seed)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1205_2107_gb300 import api, autograd, inputs

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def oracle_gradient(d, e, w, C):
    """dL/dd, dL/de from the oracle: eigenpairs by bisection + inverse
    iteration, gradient by the dense formula."""
    Wo, Zo = oracle.eigh_tridiagonal(d, e[:len(d) - 1])
    proj = np.einsum("ji,ji->i", C, Zo)
    Zbar = 2.0 * C * proj[None, :]
    return oracle.adjoint(Wo, Zo, w, Zbar, tau=0.0)


def loss_np(W, Z, w, C):
    return float(w @ W + np.sum(np.einsum("ji,ji->i", C, Z) ** 2))


def gpu_gradient_batched(ds, es, ws, Cs):
    sizes = [len(d) for d in ds]
    lay = api.BatchLayout(sizes, "cuda")
    d = _dev(np.concatenate(ds))
    e = _dev(np.concatenate(es))
    W, Z = api.eigh_tridiagonal_batched(d, e, lay)
    W, Z = W[:lay.k_total], Z[:lay.z_total]
    Wbar = _dev(np.concatenate(ws))
    # Zbar block p (column-major): column i = 2 (c_i^T z_i) c_i
    Zbar = torch.empty_like(Z)
    for p, n in enumerate(sizes):
        z0 = lay.z_offsets_host[p]
        Zp = Z[z0:z0 + n * n].view(n, n).t()  # (n, n), column i = z_i
        Cp = _dev(Cs[p])
        proj = (Cp * Zp).sum(0)
        Zbar[z0:z0 + n * n] = (2.0 * Cp * proj[None, :]).t().reshape(-1)
    dbar, ebar = api.eigh_tridiagonal_backward(W, Z, Wbar, Zbar, lay)
    out = []
    for p, n in enumerate(sizes):
        r0 = lay.offsets_host[p]
        out.append((dbar[r0:r0 + n].cpu().numpy(), ebar[r0:r0 + n - 1].cpu().numpy(),
                    ebar[r0 + n - 1].item() if n else 0.0))
    return out


def assert_close_grad(g, go, what):
    scale = max(float(np.max(np.abs(go))), 1e-300)
    err = float(np.max(np.abs(g - go))) if g.size else 0.0
    assert err <= 1e-8 * scale, f"{what}: max error {err:.3e} (scale {scale:.3e})"


def test_ragged_batch_matches_oracle_gradient():
    rng = np.random.default_rng(77)
    sizes = [2, 3, 17, 64, 65, 130, 1, 200]
    ds = [rng.standard_normal(n) for n in sizes]
    es = [np.append(rng.standard_normal(n - 1), 0.0) if n > 1 else np.zeros(1)[:n] for n in sizes]
    es = [x if len(x) == n else np.zeros(n) for x, n in zip(es, sizes)]
    ws = [rng.standard_normal(n) for n in sizes]
    Cs = [rng.standard_normal((n, n)) for n in sizes]
    got = gpu_gradient_batched(ds, es, ws, Cs)
    for (gd, ge, elast), d, e, w, C in zip(got, ds, es, ws, Cs):
        od, oe = oracle_gradient(d, e, w, C)
        assert_close_grad(gd, od, f"dbar n={len(d)}")
        if len(d) > 1:
            assert_close_grad(ge, oe, f"ebar n={len(d)}")
        assert elast == 0.0


def test_values_only_gradient_is_the_fused_pass():
    rng = np.random.default_rng(5)
    sizes = [5, 33, 100]
    lay = api.BatchLayout(sizes, "cuda")
    ds = [rng.standard_normal(n) for n in sizes]
    es = [np.append(rng.standard_normal(n - 1), 0.0) for n in sizes]
    ws = [rng.standard_normal(n) for n in sizes]
    W, Z = api.eigh_tridiagonal_batched(_dev(np.concatenate(ds)), _dev(np.concatenate(es)), lay)
    dbar, ebar = api.eigh_tridiagonal_backward(W[:lay.k_total], Z[:lay.z_total], _dev(np.concatenate(ws)), None,
                                               lay)
    for p, (d, e, w) in enumerate(zip(ds, es, ws)):
        Wo, Zo = oracle.eigh_tridiagonal(d, e[:-1])
        od, oe = oracle.adjoint(Wo, Zo, w, None)
        r0, n = lay.offsets_host[p], sizes[p]
        assert_close_grad(dbar[r0:r0 + n].cpu().numpy(), od, "dbar")
        assert_close_grad(ebar[r0:r0 + n - 1].cpu().numpy(), oe, "ebar")


def test_backward_is_deterministic():
    d, e, w, C = inputs.adjoint_case(batch=3, n=96, seed=11)
    a = gpu_gradient_batched(list(d), list(e), list(w), list(C))
    b = gpu_gradient_batched(list(d), list(e), list(w), list(C))
    for (d1, e1, _), (d2, e2, _) in zip(a, b):
        assert np.array_equal(d1, d2) and np.array_equal(e1, e2)


def test_autograd_single_problem_matches_oracle_and_finite_differences():
    rng = np.random.default_rng(1206)
    n = 48
    d_np, e_np = rng.standard_normal(n), rng.standard_normal(n - 1)
    w_np, C_np = rng.standard_normal(n), rng.standard_normal((n, n))
    d = _dev(d_np).requires_grad_(True)
    e = _dev(e_np).requires_grad_(True)
    W, Z = autograd.eigh_tridiagonal_autograd(d, e)
    w, C = _dev(w_np), _dev(C_np)
    loss = (w * W).sum() + ((C * Z).sum(0) ** 2).sum()
    loss.backward()
    od, oe = oracle_gradient(d_np, np.append(e_np, 0.0), w_np, C_np)
    assert_close_grad(d.grad.cpu().numpy(), od, "d.grad")
    assert_close_grad(e.grad.cpu().numpy(), oe, "e.grad")
    # central differences of the loss through the forward solver, h = 1e-6
    h = 1e-6
    for which, j in [("d", 0), ("d", 17), ("d", n - 1), ("e", 0), ("e", 20), ("e", n - 2)]:
        vals = []
        for s in (+1, -1):
            dd, ee = d_np.copy(), e_np.copy()
            (dd if which == "d" else ee)[j] += s * h
            Wp, Zp = api.eigh_tridiagonal(_dev(dd), _dev(np.append(ee, 0.0)))
            vals.append(loss_np(Wp.cpu().numpy(), Zp.cpu().numpy(), w_np, C_np))
        fd = (vals[0] - vals[1]) / (2 * h)
        g = (d.grad if which == "d" else e.grad)[j].item()
        assert abs(fd - g) <= 1e-6 * max(abs(g), 1.0), f"{which}[{j}]: fd {fd:.10e} vs grad {g:.10e}"


def test_full_size_adjoint_batch_sampled():
    """256 problems of n = 512 (the differentiation workload), gradients of
    sampled problems against the oracle; every problem checked for finiteness."""
    d, e, w, C = inputs.adjoint_case()
    batch, n = d.shape
    lay = api.BatchLayout([n] * batch, "cuda")
    dt = _dev(d.reshape(-1)).requires_grad_(True)
    et = _dev(e.reshape(-1)).requires_grad_(True)
    W, Z = autograd.eigh_tridiagonal_batched_autograd(dt, et, lay)
    Zb = Z.view(batch, n, n)  # [p, i, j] = Z_p(j, i): row i of the view is column i of Z_p
    Ct = _dev(C).transpose(1, 2)  # [p, i, j] = C_p(j, i)
    loss = (_dev(w).reshape(-1) * W).sum() + ((Ct * Zb).sum(2) ** 2).sum()
    loss.backward()
    gd = dt.grad.view(batch, n).cpu().numpy()
    ge = et.grad.view(batch, n).cpu().numpy()
    assert np.all(np.isfinite(gd)) and np.all(np.isfinite(ge))
    assert np.all(ge[:, -1] == 0.0)
    for p in (0, 101, 255):
        od, oe = oracle_gradient(d[p], e[p], w[p], C[p])
        assert_close_grad(gd[p], od, f"dbar problem {p}")
        assert_close_grad(ge[p, :-1], oe, f"ebar problem {p}")


def test_recompute_gives_the_same_gradient():
    """recompute=True solves again in the backward pass instead of keeping Z;
    the solver is deterministic, so the gradients agree bit for bit."""
    d, e, w, C = inputs.adjoint_case(batch=8, n=200, seed=21)
    batch, n = d.shape
    lay = api.BatchLayout([n] * batch, "cuda")
    grads = []
    for recompute in (False, True):
        dt = _dev(d.reshape(-1)).requires_grad_(True)
        et = _dev(e.reshape(-1)).requires_grad_(True)
        W, Z = autograd.eigh_tridiagonal_batched_autograd(dt, et, lay, recompute=recompute)
        Zb = Z.view(batch, n, n)
        Ct = _dev(C).transpose(1, 2)
        loss = (_dev(w).reshape(-1) * W).sum() + ((Ct * Zb).sum(2) ** 2).sum()
        loss.backward()
        grads.append((dt.grad.clone(), et.grad.clone()))
    assert torch.equal(grads[0][0], grads[1][0]) and torch.equal(grads[0][1], grads[1][1])
    # the single-problem function too
    g1 = []
    for recompute in (False, True):
        dt = _dev(d[0]).requires_grad_(True)
        et = _dev(e[0][:-1]).requires_grad_(True)
        W, Z = autograd.eigh_tridiagonal_autograd(dt, et, recompute=recompute)
        ((_dev(w[0]) * W).sum() + ((_dev(C[0]) * Z).sum(0) ** 2).sum()).backward()
        g1.append((dt.grad.clone(), et.grad.clone()))
    assert torch.equal(g1[0][0], g1[1][0]) and torch.equal(g1[0][1], g1[1][1])
