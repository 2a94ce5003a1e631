"""GPU parity of the backward pass (mrrr_backward and the autograd wrappers)
against the oracle's dense reference gradient, computed from the oracle's
own eigendecomposition, and against central finite differences of the loss
sum_i w_i lambda_i + sum_i (c_i^T z_i)^2 (w, C iid normal from a seed)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1205_2107_gb300 import api, autograd, inputs
from tests import checks

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def oracle_gradient(d, e, w, C):
    """dL/dd, dL/de from the oracle: eigenpairs by bisection + inverse
    iteration, gradient by the dense formula."""
    Wo, Zo = oracle.eigh_tridiagonal(d, e[:len(d) - 1])
    proj = np.einsum("ji,ji->i", C, Zo)
    Zbar = 2.0 * C * proj[None, :]
    return oracle.adjoint(Wo, Zo, w, Zbar, tau=api.DEFAULT_TAU_REL * float(np.max(np.abs(Wo))))


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


# Finite-difference acceptance: relative error 1e-6, plus a floor for
# entries near zero.  The floor is the rounding noise of the differenced
# loss: the solver returns each eigenpair to a few ulps, so the loss of a
# 512 x 512 problem (magnitude up to ~1e3) carries noise of ~1e-13, which
# the central difference divides by 2h = 2e-6.
FD_RTOL = 1e-6
FD_FLOOR = 1e-7


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
    # central differences of the loss through the forward solver, h = 1e-6,
    # with Richardson's control: an entry whose differences at h and h/2
    # disagree by more than 1e-6 relative is not resolved by differencing at
    # this step (small gaps) and rests on the oracle comparison above
    h = 1e-6
    resolved = 0
    for which, j in [("d", 0), ("d", 17), ("d", n - 1), ("e", 0), ("e", 20), ("e", n - 2)]:
        fds = []
        for step in (h, h / 2):
            vals = []
            for s in (+1, -1):
                dd, ee = d_np.copy(), e_np.copy()
                (dd if which == "d" else ee)[j] += s * step
                Wp, Zp = api.eigh_tridiagonal(_dev(dd), _dev(np.append(ee, 0.0)))
                vals.append(loss_np(Wp.cpu().numpy(), Zp.cpu().numpy(), w_np, C_np))
            fds.append((vals[0] - vals[1]) / (2 * step))
        g = (d.grad if which == "d" else e.grad)[j].item()
        if abs(fds[0] - fds[1]) > FD_RTOL * abs(fds[0]) + FD_FLOOR:
            continue
        resolved += 1
        assert abs(fds[0] - g) <= FD_RTOL * abs(g) + FD_FLOOR, f"{which}[{j}]: fd {fds[0]:.10e} vs grad {g:.10e}"
    assert resolved >= 4


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


def test_finite_differences_on_the_adjoint_workload():
    """Central differences (h = 1e-6) of the loss along 8 seeded random
    directions in (d, e) for four problems of the 256 x 512 workload, against
    the directional derivative g . v of the backward pass.  Richardson's
    control: a direction whose differences at h and h/2 disagree by more than
    1e-6 relative (tiny gaps make the loss strongly curved there) is counted
    as unresolved and rests on the oracle comparison of the full-batch test."""
    d, e, w, C = inputs.adjoint_case()
    batch, n = d.shape
    probs = [0, 37, 128, 255]
    # gradients of the four problems (a batch of four through the C ABI)
    grads = gpu_gradient_batched([d[p] for p in probs], [e[p] for p in probs], [w[p] for p in probs],
                                 [C[p] for p in probs])
    rng = np.random.default_rng(1206)
    h = 1e-6
    cases, ds, es = [], [], []
    for k, p in enumerate(probs):
        for _ in range(8):
            vd = rng.standard_normal(n)
            ve = rng.standard_normal(n)
            ve[-1] = 0.0
            gdot = float(grads[k][0] @ vd + grads[k][1] @ ve[:-1])
            cases.append((p, gdot))
            for step in (h, -h, h / 2, -h / 2):
                ds.append(d[p] + step * vd)
                es.append(e[p] + step * ve)
    lay = api.BatchLayout([n] * len(ds), "cuda")
    W, Z = api.eigh_tridiagonal_batched(_dev(np.concatenate(ds)), _dev(np.concatenate(es)), lay)
    Ws, Zs = lay.unpack(W, Z)
    losses = []
    for q in range(len(ds)):
        p = cases[q // 4][0]
        losses.append(loss_np(Ws[q].cpu().numpy(), Zs[q].cpu().numpy(), w[p], C[p]))
    resolved = 0
    worst = 0.0
    for c, (p, gdot) in enumerate(cases):
        lp, lm, lp2, lm2 = losses[4 * c:4 * c + 4]
        fd1 = (lp - lm) / (2 * h)
        fd2 = (lp2 - lm2) / h
        if abs(fd1 - fd2) > FD_RTOL * abs(fd1) + FD_FLOOR:
            continue
        resolved += 1
        err = abs(fd1 - gdot) / max(abs(gdot), 1e-300)
        worst = max(worst, err)
        assert abs(fd1 - gdot) <= FD_RTOL * abs(gdot) + FD_FLOOR, f"problem {p}: fd {fd1:.12e} vs g.v {gdot:.12e}"
    print(f"finite differences: {resolved}/{len(cases)} directions resolved, worst relative error {worst:.2e}")
    assert resolved >= len(cases) // 4


def test_degenerate_spectrum_gradient_glued():
    """Glued W21+ x20 (n = 420): groups of 20 eigenvalues, many equal to the
    last bit.  For a loss that depends on T alone -- weights constant on each
    group and, per group, the squared norm of the projection of one vector
    c_G onto the group's invariant subspace -- the gradient is defined even
    though individual vectors are not; the backward pass must give it finite
    and equal to the oracle's dense formula at the same threshold.  At
    tau = 1e-8 ||T|| every within-group pair is dropped and the two agree to
    1e-8 relative; at the default threshold (64 eps ||T||) pairs with tiny
    gaps are kept, whose terms F = 1/gap amplify rounding, and the two must
    agree within that amplification (4 n eps max|Z^T Zbar| / smallest kept
    gap per kept pair)."""
    d_np, e_np = inputs.glued_wilkinson(20)
    n = len(d_np)
    lay = api.BatchLayout([n], "cuda")
    dt, et = _dev(d_np), _dev(np.append(e_np, 0.0))
    W, Z = api.eigh_tridiagonal_batched(dt, et, lay)
    W, Z = W[:n], Z[:n * n]
    Wo, Zo = oracle.eigh_tridiagonal(d_np, e_np)
    tn = float(np.max(np.abs(Wo)))
    groups = checks.groups_by_gap(Wo, 1e-6 * tn)
    rng = np.random.default_rng(420)
    wv = np.zeros(n)
    Cg = np.zeros((n, n))  # column i = c_G of the group of i
    for a, b in groups:
        wv[a:b] = rng.standard_normal()
        Cg[:, a:b] = rng.standard_normal(n)[:, None]

    def zbar_of(Zm):
        proj = np.einsum("ji,ji->i", Cg, Zm)
        return 2.0 * Cg * proj[None, :]

    Zg = Z.view(n, n).t().cpu().numpy()
    for tau_rel in (1e-8, api.DEFAULT_TAU_REL):
        Zbar = _dev(zbar_of(Zg).T.reshape(-1).copy())
        dbar, ebar = api.eigh_tridiagonal_backward(W, Z, _dev(wv), Zbar, lay, tau_rel=tau_rel)
        gd, ge = dbar[:n].cpu().numpy(), ebar[:n - 1].cpu().numpy()
        assert np.all(np.isfinite(gd)) and np.all(np.isfinite(ge))
        od, oe = oracle.adjoint(Wo, Zo, wv, zbar_of(Zo), tau=tau_rel * tn)
        scale = max(np.max(np.abs(od)), np.max(np.abs(oe)))
        if tau_rel == 1e-8:
            tol = 1e-8 * scale
        else:
            tau = tau_rel * tn
            gaps = np.abs(Wo[None, :] - Wo[:, None])
            kept = (gaps > tau) & (gaps < 1e-6 * tn)
            G = np.abs(Zo.T @ zbar_of(Zo)).max()
            tol = 1e-8 * scale + (np.sqrt(kept.sum()) * 4 * n * checks.EPS * G / gaps[kept].min() if kept.any() else 0.0)
        err = max(np.max(np.abs(gd - od)), np.max(np.abs(ge - oe)))
        assert err <= tol, f"tau_rel={tau_rel:.2e}: gradient error {err:.3e} > {tol:.3e}"

