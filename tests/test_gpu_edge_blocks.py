"""GPU parity on split structures and magnitudes that broke the first oracle:
a cluster of one block with another block's eigenvalue between its members,
tiny blocks beside normal ones, a small block beside a large entry, and a
seeded sample of small structured tridiagonals (exact zeros in e, repeated
entries, entries spread over 60 binades, scalings 2^-400 and 2^400)."""
import numpy as np
import pytest

import oracle
from paper_1205_2107_gb300 import inputs
from tests.test_gpu_solver import assert_parity

pytestmark = pytest.mark.gpu


def test_cluster_members_separated_by_another_block():
    d0, e0 = inputs.wilkinson_plus(21)
    W0 = np.linalg.eigvalsh(oracle.tridiag_dense(d0, e0))
    lo, hi = W0[17], W0[18]
    d = np.append(d0, lo + (hi - lo) / 2)
    e = np.append(e0, 0.0)
    assert_parity(d, e)


def test_glued_copies_with_blocks_inside_their_clusters():
    """Five glued W21+ copies (clusters of 5) and, as separate 1x1 blocks,
    the midpoints of the top cluster."""
    dg, eg = inputs.glued_wilkinson(5)
    W0 = oracle.eigvalsh_tridiagonal(dg, eg)
    top = W0[-5:]
    mids = top[:-1] + np.diff(top) / 2
    d = np.concatenate([dg, mids])
    e = np.concatenate([eg, np.zeros(len(mids))])
    assert_parity(d, e)


def test_tiny_block_beside_a_normal_one():
    assert_parity(np.array([1.0, 2.23341364e-239, 0.0]), np.zeros(2))


def test_small_block_beside_a_large_entry():
    assert_parity(np.array([0.0, 0.0, 512.0, 0.0, 0.0]), np.array([0.0, 0.0, 0.0, 1.0]))


def _structured(rng):
    n = int(rng.integers(1, 41))

    def entries(k):
        kind = rng.integers(0, 4, size=k)
        x = np.where(kind == 0, 0.0, 0.0)
        x = np.where(kind == 1, rng.choice([1.0, -1.0, 0.5, 2.0], size=k), x)
        x = np.where(kind == 2, rng.uniform(-4, 4, size=k), x)
        x = np.where(kind == 3, rng.uniform(0.5, 1.0, size=k) * np.exp2(rng.integers(-30, 31, size=k)), x)
        return x

    scale = np.exp2(float(rng.choice([0, 0, -400, 400])))
    return entries(n) * scale, entries(n - 1) * scale


@pytest.mark.parametrize("seed", range(40))
def test_structured_sample(seed):
    d, e = _structured(np.random.default_rng(7000 + seed))
    assert_parity(d, e)
