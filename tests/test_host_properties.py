"""Property-based checks of the host-side batch packing (CPU only; needs
hypothesis): offsets are prefix sums of the sizes, every problem's W and Z
blocks are disjoint and cover the packed buffers, unpack returns views of
the right shapes at the right places, and invalid ranges are refused."""
import numpy as np
import pytest
import torch

from paper_1205_2107_gb300.api import BatchLayout

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings


@st.composite
def layouts(draw):
    sizes = draw(st.lists(st.integers(0, 40), min_size=0, max_size=12))
    subset = draw(st.booleans())
    if not subset:
        return sizes, None, None
    il, iu = [], []
    for n in sizes:
        if n == 0:
            il.append(1), iu.append(0)
            continue
        a = draw(st.integers(1, n))
        il.append(a), iu.append(draw(st.integers(a, n)))
    return sizes, il, iu


@settings(max_examples=200, deadline=None, derandomize=True)
@given(layouts())
def test_packing(case):
    sizes, il, iu = case
    lay = BatchLayout(sizes, "cpu", il, iu)
    ks = [0 if n == 0 else (n if il is None else iu[p] - il[p] + 1) for p, n in enumerate(sizes)]
    assert lay.offsets_host == [0] + np.cumsum(sizes, dtype=np.int64).tolist()
    assert lay.w_offsets_host == [0] + np.cumsum(ks, dtype=np.int64).tolist()
    assert lay.z_offsets_host == [0] + np.cumsum([n * k for n, k in zip(sizes, ks)], dtype=np.int64).tolist()
    assert lay.n_total == sum(sizes) and lay.k_total == sum(ks) and lay.n_max == max(sizes, default=0)
    assert lay.all == (il is None or all(a == 1 and b == n for n, a, b in zip(sizes, il, iu)))
    W = torch.arange(lay.k_total, dtype=torch.float64)
    Z = torch.arange(lay.z_total, dtype=torch.float64)
    Ws, Zs = lay.unpack(W, Z)
    seen = torch.zeros(lay.z_total, dtype=torch.int64)
    for p, (n, k) in enumerate(zip(sizes, ks)):
        assert Ws[p].numel() == k and tuple(Zs[p].shape) == (n, k)
        if n and k:
            # column-major n x k block: Z_p[i, j] = Z[z0 + j n + i]
            z0 = lay.z_offsets_host[p]
            assert Zs[p][n - 1, k - 1].item() == z0 + (k - 1) * n + n - 1
            seen[z0:z0 + n * k] += 1
    assert torch.all(seen == 1)


@pytest.mark.parametrize("sizes,il,iu", [([5], [0], [3]), ([5], [2], [6]), ([5], [4], [3]), ([5, 3], [1], [5]),
                                         ([-1], None, None)])
def test_invalid_ranges_are_refused(sizes, il, iu):
    with pytest.raises(ValueError):
        BatchLayout(sizes, "cpu", il, iu)
