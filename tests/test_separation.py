"""The oracle and the CUDA path stay apart, and the product path has no CPU
fallback (CPU only: the checks read sources and call the Python binding with
CPU tensors, which it must refuse before any library call)."""
import ast
import os
import re

import numpy as np
import pytest
import torch

from paper_1205_2107_gb300 import api, autograd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1205_2107_gb300")


def _py_files(folder):
    for dirpath, _, files in os.walk(folder):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def _imported_roots(tree):
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name.split(".")[0], node
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            yield node.module.split(".")[0], node


def test_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        tree = ast.parse(open(path).read())
        roots = {r for r, _ in _imported_roots(tree)}
        assert "oracle" not in roots, path
        # no indirect route either (importlib, __import__ with a name string)
        names = {n.value for n in ast.walk(tree) if isinstance(n, ast.Constant) and isinstance(n.value, str)}
        assert not any(v == "oracle" or v.startswith("oracle.") for v in names), path


def test_oracle_never_imports_the_package():
    for path in _py_files(os.path.join(ROOT, "oracle")):
        roots = {r for r, _ in _imported_roots(ast.parse(open(path).read()))}
        assert not roots & {"paper_1205_2107_gb300", "torch", "bench"}, path


def test_sources_share_no_header():
    """The C oracle includes only system headers; the CUDA sources include
    only their own headers and the public ABI header."""
    c_incl = re.findall(r'#include\s*([<"][^>"]+[>"])', open(os.path.join(ROOT, "oracle", "oracle.c")).read())
    assert c_incl and all(h.startswith("<") for h in c_incl), c_incl
    csrc = os.path.join(PKG, "csrc")
    own = set(os.listdir(csrc))
    for f in sorted(own):
        for h in re.findall(r'#include\s*"([^"]+)"', open(os.path.join(csrc, f)).read()):
            assert os.path.basename(h) in own or h == "../../include/mrrr.h", (f, h)
            assert "oracle" not in h, (f, h)


def test_bench_runs_the_oracle_only_in_its_cpu_legs():
    """bench.py imports the oracle inside the oracle sampler, the reference
    arm, and the cpu_baseline block of its own arm, nowhere else."""
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    top = {r for r, node in _imported_roots(ast.Module(body=tree.body, type_ignores=[]))
           if node in tree.body}
    assert "oracle" not in top
    where = []
    for fn in ast.walk(tree):
        if not isinstance(fn, ast.FunctionDef):
            continue
        for stmt in ast.walk(fn):
            if isinstance(stmt, ast.If) and any(r == "oracle" for r, _ in _imported_roots(
                    ast.Module(body=stmt.body, type_ignores=[]))):
                where.append((fn.name, ast.unparse(stmt.test)))
        for r, _ in _imported_roots(fn):
            if r == "oracle":
                where.append((fn.name, None))
    names = {w[0] for w in where}
    assert names == {"oracle_sample", "run_reference", "run_ours"}, where
    guards = [test for name, test in where if name == "run_ours" and test is not None]
    assert guards and all("no_cpu_baseline" in g and "world == 1" in g for g in guards), guards


def _cpu(*shape):
    return torch.zeros(*shape, dtype=torch.float64)


def test_public_calls_refuse_cpu_tensors():
    """No CPU fallback: every entry point of the binding raises on host
    tensors instead of computing the result some other way."""
    d, e = _cpu(8), _cpu(8)
    with pytest.raises(TypeError, match="CUDA tensor"):
        api.eigh_tridiagonal(d, e)
    with pytest.raises(TypeError, match="CUDA tensor"):
        api.eigh_tridiagonal(d, e, 2, 3, vectors=False)
    lay = api.BatchLayout([3, 5], "cpu")
    with pytest.raises(TypeError, match="CUDA tensor"):
        api.eigh_tridiagonal_batched(d, e, lay)
    with pytest.raises(TypeError, match="CUDA tensor"):
        api.eigh_tridiagonal_backward(_cpu(8), _cpu(34), _cpu(8), None, lay)
    with pytest.raises(TypeError, match="CUDA tensor"):
        autograd.eigh_tridiagonal_autograd(d.clone().requires_grad_(True), e[:7].clone())
    with pytest.raises(TypeError, match="CUDA tensor"):
        autograd.eigh_tridiagonal_batched_autograd(d.clone().requires_grad_(True), e.clone(), lay)
    with pytest.raises(TypeError, match="CUDA tensor"):
        api.autotune_batched(d, e, lay)
    with pytest.raises(TypeError, match="CUDA tensor"):
        api.eigh_tridiagonal(np.zeros(8), np.zeros(7))


def test_dense_slice_and_shard_calls_refuse_cpu_tensors():
    """The same for the dense stages, the index slices and the sharded
    driver."""
    from paper_1205_2107_gb300 import shard
    A, d = torch.eye(4, dtype=torch.float64), _cpu(8)
    calls = [lambda: api.tridiagonalize(A), lambda: api.apply_q(A, _cpu(2), A), lambda: api.eigh_dense(A),
             lambda: api.eigh_dense(A, 1, 2, vectors=False), lambda: api.cholesky(A),
             lambda: api.eigh_generalized(A, A), lambda: api.eigh_tridiagonal_slice(d, d, None, None, 2, 0),
             lambda: shard.eigh_tridiagonal_sharded(d, d)]
    for call in calls:
        with pytest.raises(TypeError, match="CUDA tensor"):
            call()


def test_a_missing_library_raises(monkeypatch):
    """Without libmrrr.so the binding raises; nothing else computes."""
    from paper_1205_2107_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib._build, "LIB", os.path.join(ROOT, "no_such_dir", "libmrrr.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def test_empty_problem_still_needs_a_device_tensor():
    with pytest.raises(TypeError, match="CUDA tensor"):
        api.eigh_tridiagonal(_cpu(0), _cpu(0))
