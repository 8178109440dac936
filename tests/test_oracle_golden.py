"""Counts printed in the paper (tests/golden/paper_counts.txt) against the oracle."""
import itertools
import os

import numpy as np

from oracle import directions, m2l

HERE = os.path.dirname(__file__)


def _rows():
    for line in open(os.path.join(HERE, "golden", "paper_counts.txt")):
        line = line.split("#")[0].strip()
        if line:
            name, arg, val = line.split()
            yield name, int(arg.split("=")[1]), int(val)


def test_paper_counts():
    seen = set()
    for name, arg, val in _rows():
        seen.add(name)
        if name == "directions":
            assert len(directions.directions(arg)) == val
        elif name == "hadamard":
            p = arg
            g = m2l.spectrum(1.0, 1.0, p, 2 * p - 1, (2, 1, 0))
            assert g.size == val
        elif name == "alpha_terms":
            assert sum(1 for a in itertools.product((0, 1), repeat=2 * arg) if any(a)) == val
    assert seen == {"directions", "hadamard", "alpha_terms"}


def test_lemma1_bound_on_equispaced_nodes():
    """Lemma 1 (Sec. 3.1): omega_L <= (2a/(L-1))^L / (4L) for L equispaced nodes on [-a, a]."""
    from math import factorial
    from oracle.interp import nodes1d
    a = 1.0
    x = np.linspace(-a, a, 200001)
    for L in range(2, 9):
        nodes = -a + 2 * a * nodes1d(L)
        omega = np.max(np.abs(np.prod(x[:, None] - nodes[None, :], axis=1))) / factorial(L)
        assert omega <= (2 * a / (L - 1)) ** L / (4 * L) * (1 + 1e-12)
