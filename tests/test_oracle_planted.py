"""The tridiagonal oracle's pins catch plausible mistakes in its C code
(CPU only).

Each case copies oracle/oracle.c, plants one mistake of the kind a careful
reader could still make -- a flipped sign in the Sturm recurrence, an index
off by one, a dropped term of the banded LU, a skipped Gram-Schmidt pass, a
wrong split row, a Jacobi rotation with the wrong angle -- compiles the copy
with the oracle's own flags and runs a battery of the pins against it in a
child process (so that a mistake that crashes the copy cannot take the test
run down).  The battery holds only checks fixed outside the oracle: the 1-2-1
Toeplitz and Clement closed forms, LAPACK's tridiagonal eigenvalues, residual
and orthogonality against the accuracy goals (paper Sec. 2.3, Eqs. Tresnorm
and Torthogo), Sturm counts between LAPACK's separated eigenvalues, and
subspaces of LAPACK's eigenvectors.  The unchanged copy must pass every
check; every planted mistake must fail at least one.  The same is done for
the Python layer (oracle/oracle.py: the power-of-two scaling and the layout
of the C library's results) and for the dense stages (oracle/dense.py,
against NumPy's and SciPy's LAPACK routines and the stages' defining
identities) on a copy of the whole oracle package.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
EPS = 2.0 ** -53

# (name, text in oracle.c, replacement): each text occurs exactly once
MISTAKES = [
    ("sturm recurrence sign", "q = (d[i] - x) - e2[i - 1] / q;", "q = (d[i] - x) + e2[i - 1] / q;"),
    ("sturm first pivot sign", "double q = d[0] - x;", "double q = x - d[0];"),
    ("block bisection index off by one",
     "if (sturm_count_block(b->m, b->d, b->e2, mid, b->pivmin) >= k)",
     "if (sturm_count_block(b->m, b->d, b->e2, mid, b->pivmin) > k)"),
    ("k-th eigenvalue index off by one", "if (cnt >= k)", "if (cnt > k)"),
    ("sturm count of a split T keeps only the last block",
     "total += sturm_count_block(m, d + s, blk.e2, x, blk.pivmin);",
     "total = sturm_count_block(m, d + s, blk.e2, x, blk.pivmin);"),
    ("split block starts one row early", "starts[nb++] = i + 1;", "starts[nb++] = i;"),
    ("blocks' eigenvalues not merged in order", "    qsort(all, nitems, sizeof(eig_t), eig_cmp);\n", ""),
    ("LU elimination sign", "w0 = a1 - mk * w1;", "w0 = a1 + mk * w1;"),
    ("LU back substitution drops the second superdiagonal",
     "    if (k + 2 < m) v -= f->u2[k] * x[k + 2];\n", ""),
    ("inverse iteration shift sign", "lu_factor(&f, d, es, mu, tiny);", "lu_factor(&f, d, es, -mu, tiny);"),
    ("Gram-Schmidt adds the projection", "for (int i = 0; i < m; ++i) x[i] -= h * v[i];",
     "for (int i = 0; i < m; ++i) x[i] += h * v[i];"),
    ("no Gram-Schmidt inside clusters", "for (int pass = 0; pass < 2; ++pass)", "for (int pass = 0; pass < 0; ++pass)"),
    ("cluster rule inverted", "q->value - p->value <= orfac * bnorm[q->block]",
     "q->value - p->value > orfac * bnorm[q->block]"),
    ("vectors not normalised", "for (int i = 0; i < m; ++i) out[i] = x[i] / nx;",
     "for (int i = 0; i < m; ++i) out[i] = x[i];"),
    ("Jacobi angle sign", "double theta = (aqq - app) / (2.0 * apq);", "double theta = (app - aqq) / (2.0 * apq);"),
    ("Jacobi rotation of V", "V[q * n + k] = s * vkp + c * vkq;", "V[q * n + k] = s * vkp - c * vkq;"),
]


def run_battery(lib_path=None):
    """The pins, run on the oracle (its library replaced by lib_path when
    given); returns the names of the checks that failed (NaN fails every
    comparison)."""
    import numpy as np
    import scipy.linalg

    import oracle.oracle as om
    from paper_1205_2107_gb300 import inputs

    if lib_path is not None:
        om.build = lambda force=False: lib_path
        om._lib = None
    failed = []

    def check(name, ok):
        if not bool(ok):
            failed.append(name)

    def dense(d, e):  # T from its definition, not through the oracle
        return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)

    def pairs(name, d, e, il=None, iu=None):
        n = len(d)
        ref = scipy.linalg.eigvalsh_tridiagonal(d, e)
        tn = float(np.max(np.abs(ref)))
        W, Z = om.eigh_tridiagonal(d, e, il, iu)
        lo, hi = (0, n) if il is None else (il - 1, iu)
        check(name + " shapes", W.shape == (hi - lo,) and Z.shape == (n, hi - lo))
        if W.shape != (hi - lo,) or Z.shape != (n, hi - lo):
            return
        check(name + " values (LAPACK)", np.max(np.abs(W - ref[lo:hi])) <= 4 * n * EPS * tn)
        R = dense(d, e) @ Z - Z * W[None, :]
        check(name + " residual", np.max(np.linalg.norm(R, axis=0)) <= 20 * n * EPS * tn)
        check(name + " orthogonality", np.max(np.abs(Z.T @ Z - np.eye(Z.shape[1]))) <= 20 * n * EPS)

    # 1-2-1 Toeplitz: eigenvalues and sine eigenvectors in closed form
    n = 64
    d, e = inputs.toeplitz(n)
    lam = inputs.toeplitz_eigenvalues(n)
    W, Z = om.eigh_tridiagonal(d, e)
    check("toeplitz values", np.max(np.abs(W - lam)) <= 4 * n * EPS * np.max(np.abs(lam)))
    j = np.arange(1, n + 1)
    k = np.arange(1, n + 1)
    S = np.sin(np.outer(j, k) * np.pi / (n + 1))
    S = S[:, np.argsort(2.0 - 2.0 * np.cos(k * np.pi / (n + 1)))]
    S /= np.linalg.norm(S, axis=0)
    check("toeplitz vectors", np.min(np.abs(np.sum(S * Z, axis=0))) >= 1.0 - 1e-10)
    # Clement: integer spectrum
    n = 51
    d, e = inputs.clement(n)
    check("clement values", np.max(np.abs(om.eigvalsh_tridiagonal(d, e) - inputs.clement_eigenvalues(n)))
          <= 4 * n * EPS * (n - 1))
    # LAPACK, residual and orthogonality: random, Wilkinson pairs, glued groups
    pairs("uniform", *inputs.uniform(200, 7))
    pairs("wilkinson W+ 201", *inputs.wilkinson_plus(201))
    pairs("glued W21+ x20", *inputs.glued_wilkinson(20))
    # a T that splits in three blocks: all, a subset, counts, single eigenvalues
    d, e = inputs.uniform(120, 9)
    e = e.copy()
    e[39] = 0.0
    e[84] = 0.0
    pairs("split", d, e)
    pairs("split subset", d, e, 30, 70)
    ref = scipy.linalg.eigvalsh_tridiagonal(d, e)
    tn = float(np.max(np.abs(ref)))
    sep = [i for i in range(0, 119, 5) if ref[i + 1] - ref[i] > 1e-8]
    check("sturm counts (split)", all(om.sturm_count(d, e, 0.5 * (ref[i] + ref[i + 1])) == i + 1 for i in sep))
    check("k-th eigenvalue (split)",
          all(abs(om.kth_eigenvalue(d, e, kk) - ref[kk - 1]) <= 4 * 120 * EPS * tn for kk in (1, 17, 60, 120)))
    # one cluster's vectors: the subspace of W+'s largest pair
    d, e = inputs.wilkinson_plus(201)
    wref, zref = scipy.linalg.eigh_tridiagonal(d, e, select="i", select_range=(199, 200))
    Zc = om.cluster_vectors(d, e, wref)
    sv = np.linalg.svd(zref.T @ Zc, compute_uv=False)
    check("cluster vectors subspace", np.min(sv) >= 1.0 - 1e-10 and np.max(sv) <= 1.0 + 1e-10)
    # Jacobi against LAPACK's dense solver
    n = 17
    d, e = inputs.uniform(n, 3)
    T = dense(d, e)
    Wj, V = om.jacobi(d, e)
    ref = np.linalg.eigvalsh(T)
    tn = float(np.max(np.abs(ref)))
    check("jacobi values", np.max(np.abs(Wj - ref)) <= 4 * n * EPS * tn)
    check("jacobi vectors", np.max(np.linalg.norm(T @ V - V * Wj[None, :], axis=0)) <= 20 * n * EPS * tn
          and np.max(np.abs(V.T @ V - np.eye(n))) <= 20 * n * EPS)
    return failed


def _compile(text, out):
    src = out[:-3] + ".c"
    with open(src, "w") as f:
        f.write(text)
    # the flags oracle.build uses
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                    "-fno-fast-math", "-o", out, src, "-lm"], check=True)
    return out


def _battery_in_child(lib_path=None, pkg_root=None, battery="run_battery"):
    """A battery (run_battery or run_dense_battery) in a child process; with
    pkg_root, ``import oracle`` finds the copy of the oracle package there."""
    paths = [p for p in (pkg_root, ROOT) if p]
    args = "%r" % (lib_path,) if battery == "run_battery" else ""
    code = ("import json, sys; sys.path[:0] = %r; "
            "from tests.test_oracle_planted import %s; "
            "print(json.dumps(%s(%s)))" % (paths, battery, battery, args))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300, cwd=ROOT)
    if r.returncode != 0:
        return None, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), ""


def _source():
    with open(SRC) as f:
        return f.read()


def test_unchanged_oracle_passes_the_battery(tmp_path):
    failed, err = _battery_in_child(_compile(_source(), str(tmp_path / "liboracle_ok.so")))
    assert failed == [], (failed, err)


@pytest.mark.parametrize("name,old,new", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    text = _source()
    assert text.count(old) == 1, "the planted text must occur exactly once in oracle.c"
    lib = _compile(text.replace(old, new), str(tmp_path / "liboracle_planted.so"))
    failed, err = _battery_in_child(lib)
    # a copy that crashes has failed too; otherwise at least one pin must fail
    assert failed is None or len(failed) > 0, name


# mistakes in the Python layer of the oracle (oracle/oracle.py): the power-of-
# two scaling and the layout of what the C library returns
PY_MISTAKES = [
    ("eigenvalues not scaled back", "return np.ldexp(W[:k], -s), Zf[:k, :n].T.copy()",
     "return np.ldexp(W[:k], s), Zf[:k, :n].T.copy()"),
    ("Z returned transposed", "return np.ldexp(W[:k], -s), Zf[:k, :n].T.copy()",
     "return np.ldexp(W[:k], -s), Zf[:k, :n].copy()"),
    ("Sturm count at an unscaled x", "float(np.ldexp(float(x), k))", "float(x)"),
    ("k-th eigenvalue not scaled back", "_load().oracle_kth_eigenvalue(n, _ptr(d), _ptr(eb), int(k)), -s)",
     "_load().oracle_kth_eigenvalue(n, _ptr(d), _ptr(eb), int(k)), s)"),
    ("cluster shifts not scaled", "mus = np.ldexp(_f64(mus), s)", "mus = _f64(mus)"),
    ("Jacobi V returned transposed", "return np.ldexp(W, -s), V.T.copy()", "return np.ldexp(W, -s), V.copy()"),
]


def _package_copy(dst, old=None, new=None, module="oracle.py"):
    import shutil
    pkg = os.path.join(dst, "oracle")
    os.makedirs(pkg)
    for name in ("__init__.py", "oracle.py", "oracle.c", "dense.py"):
        shutil.copy(os.path.join(ROOT, "oracle", name), pkg)
    if old is not None:
        path = os.path.join(pkg, module)
        with open(path) as f:
            text = f.read()
        assert text.count(old) == 1, "the planted text must occur exactly once in " + module
        with open(path, "w") as f:
            f.write(text.replace(old, new))
    return dst


def test_unchanged_oracle_package_passes_the_battery(tmp_path):
    failed, err = _battery_in_child(pkg_root=_package_copy(str(tmp_path)))
    assert failed == [], (failed, err)


@pytest.mark.parametrize("name,old,new", PY_MISTAKES, ids=[m[0] for m in PY_MISTAKES])
def test_planted_python_mistake_fails_a_pin(tmp_path, name, old, new):
    failed, err = _battery_in_child(pkg_root=_package_copy(str(tmp_path), old, new))
    assert failed, (name, err)  # the battery runs through and records a failed pin


def run_dense_battery():
    """The dense oracle's pins (oracle/dense.py, paper Sec. 1.2 stages 1-6)
    against NumPy's and SciPy's LAPACK routines and the defining identities;
    returns the names of the checks that failed."""
    import numpy as np
    import scipy.linalg

    from oracle import dense as od

    failed = []

    def check(name, ok):
        if not bool(ok):
            failed.append(name)

    rng = np.random.default_rng(1205)
    n = 40
    X = rng.standard_normal((n, n))
    A = (X + X.T) / 2
    G = rng.standard_normal((n, n))
    B = G @ G.T + n * np.eye(n)
    an = float(np.linalg.norm(A, 2))
    tol = 1e-12
    # a reflector maps x onto beta e_1, with beta of the sign opposite to x_0
    x = rng.standard_normal(7)
    v, tau, beta = od.householder_vector(x)
    H = np.eye(7) - tau * np.outer(v, v)
    e1 = np.zeros(7)
    e1[0] = 1.0
    check("reflector maps onto e_1", v[0] == 1.0 and np.max(np.abs(H @ x - beta * e1)) <= tol * np.linalg.norm(x))
    check("reflector sign", abs(beta + np.sign(x[0]) * np.linalg.norm(x)) <= tol * np.linalg.norm(x))
    # stage 3: Q^T A Q = T with Q orthogonal, T's eigenvalues LAPACK's
    d, e, V, tau = od.tridiagonal_reduction(A)
    Q = od.form_q(V, tau, n)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    ref = np.linalg.eigvalsh(A)
    check("Q orthogonal", np.max(np.abs(Q.T @ Q - np.eye(n))) <= tol)
    check("Q^T A Q = T", np.max(np.abs(Q.T @ A @ Q - T)) <= tol * an)
    check("T's eigenvalues", np.max(np.abs(np.linalg.eigvalsh(T) - ref)) <= tol * an)
    # stages 3-5: the standard problem
    W, Y = od.eigh_dense(A)
    check("dense eigenvalues", np.max(np.abs(W - ref)) <= tol * an)
    check("dense residual", np.max(np.linalg.norm(A @ Y - Y * W[None, :], axis=0)) <= tol * an)
    check("dense orthogonality", np.max(np.abs(Y.T @ Y - np.eye(n))) <= tol)
    # stage 1 and the triangular solves
    L = od.cholesky(B)
    bn = float(np.linalg.norm(B, 2))
    check("cholesky lower", np.all(np.triu(L, 1) == 0.0))
    check("cholesky is numpy's", np.max(np.abs(L - np.linalg.cholesky(B))) <= tol * np.sqrt(bn))
    R = rng.standard_normal((n, 3))
    Lr = np.linalg.cholesky(B)
    check("forward substitution", np.max(np.abs(Lr @ od.forward_substitution(Lr, R) - R)) <= tol * bn)
    check("back substitution", np.max(np.abs(Lr.T @ od.back_substitution_transposed(Lr, R) - R)) <= tol * bn)
    # stage 2: C = L^-1 A L^-T against SciPy's triangular solves
    C = od.reduce_generalized(A, Lr)
    M = scipy.linalg.solve_triangular(Lr, A, lower=True)
    Cref = scipy.linalg.solve_triangular(Lr, M.T, lower=True)
    check("reduction to standard form", np.max(np.abs(C - Cref)) <= tol * an)
    # stages 1-6: the pencil
    Wg, Xg = od.eigh_generalized(A, B)
    wref = scipy.linalg.eigh(A, B, eigvals_only=True)
    check("pencil eigenvalues", np.max(np.abs(Wg - wref)) <= tol * an)
    check("A X = B X Lambda", np.max(np.abs(A @ Xg - (B @ Xg) * Wg[None, :])) <= tol * an)
    check("X^T B X = I", np.max(np.abs(Xg.T @ B @ Xg - np.eye(n))) <= tol * n)
    return failed


# mistakes in the dense oracle (oracle/dense.py)
DENSE_MISTAKES = [
    ("reflector sign that cancels", "beta = -norm if alpha >= 0.0 else norm", "beta = norm if alpha >= 0.0 else -norm"),
    ("reflector factor sign", "tau = (beta - alpha) / beta", "tau = (alpha - beta) / beta"),
    ("two-sided update without its correction", "w = p - (0.5 * t * float(p @ v)) * v", "w = p"),
    ("reflectors applied first to last", "for k in range(V.shape[1] - 1, -1, -1):", "for k in range(V.shape[1]):"),
    ("stage 5 left out", "return W, apply_q(V, tau, Z)", "return W, Z"),
    ("Cholesky pivot without the earlier columns", "s = B[j, j] - float(L[j, :j] @ L[j, :j])", "s = B[j, j]"),
    ("Cholesky column divided by the pivot squared",
     "L[j + 1:, j] = (B[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]",
     "L[j + 1:, j] = (B[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / s"),
    ("forward substitution without the division", "X[i] = (X[i] - L[i, :i] @ X[:i]) / L[i, i]",
     "X[i] = X[i] - L[i, :i] @ X[:i]"),
    ("back substitution by rows of L instead of columns", "X[i] = (X[i] - L[i + 1:, i] @ X[i + 1:]) / L[i, i]",
     "X[i] = (X[i] - L[i, i + 1:] @ X[i + 1:]) / L[i, i]"),
    ("second solve of stage 2 without the transpose", "C = forward_substitution(L, M.T)",
     "C = forward_substitution(L, M)"),
    ("stage 6 by L^-1 instead of L^-T", "return W, back_substitution_transposed(L, Y)",
     "return W, forward_substitution(L, Y)"),
]


def test_unchanged_dense_oracle_passes_the_battery(tmp_path):
    failed, err = _battery_in_child(pkg_root=_package_copy(str(tmp_path)), battery="run_dense_battery")
    assert failed == [], (failed, err)


@pytest.mark.parametrize("name,old,new", DENSE_MISTAKES, ids=[m[0] for m in DENSE_MISTAKES])
def test_planted_dense_mistake_fails_a_pin(tmp_path, name, old, new):
    failed, err = _battery_in_child(pkg_root=_package_copy(str(tmp_path), old, new, module="dense.py"),
                                    battery="run_dense_battery")
    assert failed, (name, err)
