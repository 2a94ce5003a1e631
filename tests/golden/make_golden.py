"""Writes the stored expected values of tests/golden/ from the oracle alone.

    python tests/golden/make_golden.py

wilkinson21.txt: the 21 eigenvalues of W21+ (d_i = |i - 11|, e_i = 1), the
smallest member of the Wilkinson family the paper tests on (Sec. 2.3).
glued_w21x20.txt: the 420 eigenvalues of 20 copies of W21+ glued by 1e-10.
Each file: a comment header, then one eigenvalue per line (%.17g, ascending).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1205_2107_gb300 import inputs  # noqa: E402

FIXTURES = {
    "wilkinson21.txt": ("W21+: d_i = |i - 11|, e_i = 1, n = 21", lambda: inputs.wilkinson_plus(21)),
    "glued_w21x20.txt": ("20 copies of W21+ glued by e = 1e-10, n = 420", lambda: inputs.glued_wilkinson(20)),
}


def values(name):
    d, e = FIXTURES[name][1]()
    return oracle.eigvalsh_tridiagonal(d, e)


def render(name):
    W = values(name)
    head = [f"# {FIXTURES[name][0]}",
            "# eigenvalues by the oracle (Sturm bisection on T to full accuracy), ascending",
            "# written by tests/golden/make_golden.py"]
    return "\n".join(head + [f"{w:.17g}" for w in W]) + "\n"


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return np.array([float(x) for x in f if not x.startswith("#")])


if __name__ == "__main__":
    for name in FIXTURES:
        with open(os.path.join(HERE, name), "w") as f:
            f.write(render(name))
        print("wrote", name)
