"""Stored eigenvalues (tests/golden/, written from the oracle by
make_golden.py): kept in sync with the oracle, pinned by properties that
hold independently of it, and matched by the GPU solver."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden  # noqa: E402

EPS = 2.0 ** -53


@pytest.mark.parametrize("name", sorted(make_golden.FIXTURES))
def test_fixture_matches_the_oracle(name):
    stored = make_golden.load(name)
    assert np.array_equal(stored, make_golden.values(name))


def test_wilkinson21_properties():
    W = make_golden.load("wilkinson21.txt")
    assert W.shape == (21,)
    assert abs(W.sum() - 110.0) <= 21 * 4 * EPS * 11  # trace: 2 (1 + ... + 10)
    # the large eigenvalues come in pairs that agree to many digits, and the
    # top pair is just above 10.74
    assert 10.74 < W[-1] < 10.75 and 0 < W[-1] - W[-2] < 1e-12
    assert W[-3] - W[-4] < 1e-9 and W[-2] - W[-3] > 0.5


def test_glued_copies_repeat_the_w21_spectrum():
    Wg = make_golden.load("glued_w21x20.txt")
    W = make_golden.load("wilkinson21.txt")
    assert Wg.shape == (420,)
    # each W21+ eigenvalue appears 20 times, spread by the 1e-10 glue
    for k, lam in enumerate(W):
        group = Wg[20 * k:20 * k + 20]
        assert np.max(np.abs(group - lam)) < 1e-9, k


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(make_golden.FIXTURES))
def test_gpu_matches_fixture(name):
    import torch
    from paper_1205_2107_gb300 import api
    d, e = make_golden.FIXTURES[name][1]()
    n = len(d)
    W = api.eigh_tridiagonal(torch.as_tensor(d, device="cuda"), torch.as_tensor(np.append(e, 0.0), device="cuda"),
                             vectors=False).cpu().numpy()
    stored = make_golden.load(name)
    assert np.max(np.abs(W - stored)) <= 4 * n * EPS * np.max(np.abs(stored))
