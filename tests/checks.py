"""Accuracy checks shared by the GPU tests (residual, orthogonality,
eigenvalue error, invariant-subspace angles).

The tolerances are the paper's accuracy goals (Sec. 2.3, Eqs. Tresnorm and
Torthogo) with the constants fixed for this repository:
  |lambda_j - lambda_j(oracle)| <= 4 n eps ||T||
  max_i ||T z_i - lambda_i z_i||  <= 20 n eps ||T||
  max |Z^T Z - I|                 <= 20 n eps
with eps = 2^-53 and ||T|| the spectral norm (max |lambda| from the oracle).
"""
from __future__ import annotations

import numpy as np
import torch

EPS = 2.0 ** -53


def residual_cols(d: torch.Tensor, e: torch.Tensor, W: torch.Tensor, Z: torch.Tensor) -> torch.Tensor:
    """||T z_i - lambda_i z_i||_2 per column, computed on the device (T is
    tridiagonal, so T Z is three shifted products)."""
    n = d.numel()
    TZ = d[:, None] * Z
    if n > 1:
        TZ[:-1] += e[: n - 1, None] * Z[1:]
        TZ[1:] += e[: n - 1, None] * Z[:-1]
    return torch.linalg.vector_norm(TZ - Z * W[None, :], dim=0)


def orthogonality(Z: torch.Tensor, cols: torch.Tensor | None = None) -> float:
    """max |Z^T Z - I| over all columns, or over (all x cols) when cols given."""
    k = Z.shape[1]
    if cols is None:
        G = Z.t() @ Z
        G.diagonal().sub_(1.0)
        return float(G.abs().max())
    G = Z.t() @ Z[:, cols]
    G[cols, torch.arange(cols.numel(), device=Z.device)] -= 1.0
    return float(G.abs().max())


def band_orthogonality(Z: torch.Tensor, width: int = 64, chunk: int = 2048) -> float:
    """max |z_i^T z_j - delta_ij| over |i - j| <= width (loss of orthogonality
    concentrates among neighbours in eigenvalue order)."""
    k = Z.shape[1]
    worst = 0.0
    for a in range(0, k, chunk):
        b = min(k, a + chunk)
        lo, hi = max(0, a - width), min(k, b + width)
        G = Z[:, a:b].t() @ Z[:, lo:hi]
        idx = torch.arange(a, b, device=Z.device)
        G[idx - a, idx - lo] -= 1.0
        worst = max(worst, float(G.abs().max()))
    return worst


def groups_by_gap(W: np.ndarray, thresh: float):
    """Runs of consecutive eigenvalues whose gaps are <= thresh."""
    groups, start = [], 0
    for i in range(1, len(W) + 1):
        if i == len(W) or W[i] - W[i - 1] > thresh:
            groups.append((start, i))
            start = i
    return groups


def subspace_errors(Zg: np.ndarray, Zo: np.ndarray, W: np.ndarray, tnorm: float, n: int, group_rel: float = 1e-6):
    """For each group of nearly equal eigenvalues, sin of the largest principal
    angle between the GPU and oracle invariant subspaces, and the bound
    1000 n eps ||T|| / (gap to the rest of the spectrum).  Returns a list of
    (sin_angle, bound)."""
    out = []
    groups = groups_by_gap(W, group_rel * tnorm)
    for a, b in groups:
        left = W[a] - W[a - 1] if a > 0 else np.inf
        right = W[b] - W[b - 1] if b < len(W) else np.inf
        gap = min(left, right)
        G, O = Zg[:, a:b], Zo[:, a:b]
        R = G - O @ (O.T @ G)  # component of the GPU subspace outside the oracle's
        sin = float(np.linalg.norm(R, 2))
        bound = 1000.0 * n * EPS * tnorm / gap if np.isfinite(gap) and gap > 0 else 0.0
        bound = max(bound, 100.0 * n * EPS)
        out.append((sin, min(bound, 1.0)))
    return out


def residual_frobenius(d: torch.Tensor, e: torch.Tensor, W: torch.Tensor, Z: torch.Tensor) -> float:
    """||T Z_C - Z_C diag(W_C)||_F for a block of columns (on the device)."""
    return float(torch.linalg.vector_norm(residual_cols(d, e, W, Z)))


def davis_kahan_errors(d: torch.Tensor, e: torch.Tensor, W: torch.Tensor, Z: torch.Tensor, W_exact: np.ndarray,
                       groups, tnorm: float, n: int):
    """Rigorous bound on the angle between each group's computed subspace and
    the exact invariant subspace, from the residual alone (Davis and Kahan's
    sin-theta theorem): sin(angle) <= ||T Z_C - Z_C W_C||_F / delta_C, with
    delta_C the distance from the computed values W_C to the exact eigenvalues
    outside the group (W_exact, accurate to a few n eps ||T||, widened by that
    amount).  Returns a list of (bound, tolerance) with the tolerance of
    subspace_errors."""
    out = []
    Wg = W.detach().cpu().numpy()
    margin = 8.0 * n * EPS * tnorm
    for a, b in groups:
        lo, hi = Wg[a:b].min(), Wg[a:b].max()
        left = lo - W_exact[a - 1] if a > 0 else np.inf
        right = W_exact[b] - hi if b < len(W_exact) else np.inf
        delta = min(left, right) - margin
        rf = residual_frobenius(d, e, W[a:b], Z[:, a:b])
        bound = rf / delta if delta > 0 else np.inf
        gap = min(left, right)
        tol = 1000.0 * n * EPS * tnorm / gap if np.isfinite(gap) and gap > 0 else 0.0
        out.append((bound, min(max(tol, 100.0 * n * EPS), 1.0)))
    return out


def full_orthogonality(Z: torch.Tensor, chunk: int = 4096) -> float:
    """max |Z^T Z - I| over all column pairs, by blocks of the upper triangle
    (the Gram matrix of 20,000 columns does not need to exist at once)."""
    k = Z.shape[1]
    worst = 0.0
    for a in range(0, k, chunk):
        b = min(k, a + chunk)
        G = Z[:, a:b].t() @ Z[:, a:]
        idx = torch.arange(b - a, device=Z.device)
        G[idx, idx] -= 1.0
        worst = max(worst, float(G.abs().max()))
        del G
    return worst


def subset_subspace_errors(Zg: np.ndarray, il: int, iu: int, W_all: np.ndarray, d, e, tnorm: float, n: int,
                           Zo_subset: np.ndarray, group_rel: float = 1e-6):
    """Subspace comparison for an index subset il..iu (1-based) of the
    spectrum W_all.  Groups of nearly equal eigenvalues are formed on the
    whole spectrum; a group inside the subset is compared with the oracle's
    subset vectors, and a group cut by the subset's ends is compared with the
    oracle's vectors of the whole group (the computed columns must lie in
    that group's invariant subspace).  Returns a list of (sin_angle, bound)."""
    import oracle
    out = []
    lo, hi = il - 1, iu  # 0-based half-open range of the subset
    for a, b in groups_by_gap(W_all, group_rel * tnorm):
        if b <= lo or a >= hi:
            continue
        left = W_all[a] - W_all[a - 1] if a > 0 else np.inf
        right = W_all[b] - W_all[b - 1] if b < len(W_all) else np.inf
        gap = min(left, right)
        bound = 1000.0 * n * EPS * tnorm / gap if np.isfinite(gap) and gap > 0 else 0.0
        bound = min(max(bound, 100.0 * n * EPS), 1.0)
        a2, b2 = max(a, lo), min(b, hi)
        G = Zg[:, a2 - lo:b2 - lo]
        if a >= lo and b <= hi:
            O = Zo_subset[:, a - lo:b - lo]
        else:
            O = oracle.cluster_vectors(d, e, W_all[a:b])
        R = G - O @ (O.T @ G)
        out.append((float(np.linalg.norm(R, 2)), bound))
    return out
