"""The oracle's sampled-row evaluation (used at grid sizes too large to assemble) agrees with
its global assembly, which the other oracle tests pin."""
import numpy as np
import pytest

from oracle.forms import Discretisation, masked, sampled_rows
from paper_1604_07994_gb300 import workloads as W


@pytest.mark.parametrize("form", ["tr", "sym", "grad"])
@pytest.mark.parametrize("which", ["cube", "layer"])
def test_sampled_rows_match_assembly(form, which):
    p = W.cube_inclusion(8, 4) if which == "cube" else W.top_layer(8, 8)
    d = Discretisation(p.n, p.cell_mu().ravel(), p.face)
    x = W.random_vector(p.n, 3).ravel()
    con = d.constrained()
    x[con] = 0.0
    y = (masked(d.saddle(form), con) @ x).reshape(4, -1)
    nodes = np.arange(0, d.nn, 7)
    ys = sampled_rows(p.n, p.cell_mu().ravel(), p.face, form, x, nodes)
    assert np.abs(ys - y[:, nodes]).max() <= 1e-14 * np.abs(y).max()
