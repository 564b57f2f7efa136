"""Pins of the oracle's active-set polish (crossover-lite of the paper's
pipeline, Sec. III.B) against independent vertices: the dense simplex on a
4-bus case and SciPy's HiGHS on perturbed 24-bus relaxations."""
import numpy as np
import pytest

from oracle.lp import kkt
from oracle.polish import polish
from paper_2512_06715_gb300.instances import workload
from tests.conftest import instance_lp
from tests.nondegenerate import highs_vertex, perturbed_lp

pytest.importorskip("scipy.optimize")


@pytest.mark.parametrize("seed", [0, 1])
def test_polish_recovers_the_highs_vertex(seed):
    """Polishing the HiGHS optimum reproduces it (the active set of a
    nondegenerate vertex is square and its two systems give the vertex back),
    and polishing a point near it (noise of 1e-12 of the largest entry on every
    component) snaps to the same vertex.  The perturbed relaxation keeps some
    rows with both a small dual and a small slack (margins ~1e-11 of the
    largest dual), so polish needs points that accurate."""
    lp = perturbed_lp(workload("uc24_g33_T24"), seed)
    x, y, obj = highs_vertex(lp)
    p = polish(lp, x, y)
    assert p is not None
    assert np.abs(p[0] - x).max() <= 1e-9 * np.abs(x).max()
    assert np.abs(p[1] - y).max() <= 1e-8 * np.abs(y).max()
    assert kkt(lp, *p).rel_kkt <= 1e-12
    rng = np.random.default_rng(seed)
    xn = x + 1e-12 * np.abs(x).max() * rng.standard_normal(x.size)
    yn = y + 1e-12 * np.abs(y).max() * rng.standard_normal(y.size)
    p = polish(lp, xn, yn)
    assert p is not None
    assert np.abs(p[0] - x).max() <= 1e-9 * np.abs(x).max()
    assert abs(kkt(lp, *p).primal_obj - obj) <= 1e-11 * abs(obj)


def test_polish_refuses_a_degenerate_vertex():
    """The unperturbed relaxation is degenerate at its optimum: the active set
    read off its HiGHS vertex is not square and polish returns None."""
    lp = instance_lp(workload("uc24_g33_T24"))
    x, y, _ = highs_vertex(lp)
    assert polish(lp, x, y) is None
