"""The seeded synthetic inputs follow their stated recipes: viscosity layouts, boundary faces,
viscosity tables and forcing of every workload the tests and the benchmark use (the paper's
columns and layers problems of Sec. 4.2.3-4.2.4, the three-box, top-layer, cube-inclusion,
batched and level-set workloads).  No GPU needed."""
import numpy as np

from paper_1604_07994_gb300 import workloads as W


def _resolved_on(ids, n, nc):
    """Every coarse cell of the nc^3 grid holds one id (the interface lies on its planes)."""
    r = n // nc
    b = ids.reshape(nc, r, nc, r, nc, r)
    return bool(np.all(b.min(axis=(1, 3, 5)) == b.max(axis=(1, 3, 5))))


def test_three_boxes_recipe():
    p = W.three_boxes(128, 8, contrast=1e4)
    q = W.three_boxes(128, 8, contrast=1e4)
    assert p.cell_id.shape == (128, 128, 128) and p.cell_id.dtype == np.uint8
    assert np.array_equal(p.cell_id, q.cell_id)  # seeded
    assert set(np.unique(p.cell_id)) == {0, 1}
    assert _resolved_on(p.cell_id, 128, 8)  # boxes on the 1/8 lattice
    assert np.array_equal(p.mu, [1.0, 1e4])
    assert p.face == (W.DIRICHLET,) * 6 and p.n_coarse == 8
    assert p.exact is not None  # manufactured forcing with its exact solution


def test_cube_inclusion_recipe():
    p = W.cube_inclusion(16, 4)
    ref = np.zeros((16, 16, 16), dtype=np.uint8)
    ref[4:12, 4:12, 4:12] = 1  # cell centres inside [1/4, 3/4]^3
    assert np.array_equal(p.cell_id, ref)
    assert np.array_equal(p.mu, [1.0, 10.0]) and p.face == (W.DIRICHLET,) * 6


def test_top_layer_recipe():
    p = W.top_layer(32, 8)
    k = np.arange(32)[:, None, None] * np.ones((1, 32, 32), dtype=int)
    assert np.array_equal(p.cell_id, (k >= 28).astype(np.uint8))  # z >= 7/8
    assert p.face == (W.FREESLIP,) * 4 + (W.DIRICHLET, W.TRACTION)
    assert np.array_equal(p.mu, [1.0, 1e3])
    f = p.nodal_forcing()
    assert np.all(f[0] == 0) and np.all(f[1] == 0)
    assert 0 < np.abs(f[2]).max() <= 8.0  # eight blobs of amplitude at most 1


def test_batched_instances_recipe():
    probs = W.batched_instances()
    again = W.batched_instances()
    assert len(probs) == 48
    sizes = set()
    for p, q in zip(probs, again):
        assert np.array_equal(p.cell_id, q.cell_id) and np.array_equal(p.mu, q.mu)
        assert p.n in (32, 48, 64, 96) and p.n_coarse == p.n // 8
        assert p.cell_id.shape == (p.n,) * 3
        assert _resolved_on(p.cell_id, p.n, p.n_coarse)
        assert p.mu[0] == 1.0 and 1.0 <= p.mu[1] <= 1e6
        assert p.face == (W.DIRICHLET,) * 6
        sizes.add(p.n)
    assert sizes == {32, 48, 64, 96}
    assert len({p.mu[1] for p in probs}) == 48  # independent contrasts


def test_paper_columns_and_layers_recipes():
    n = 16
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    cols = W.viscosity_columns(n)
    ref = (((x < 0.25) & (y < 0.25)) | ((x > 0.75) & (y > 0.75))).astype(np.uint8)
    assert np.array_equal(cols.cell_id, ref)
    assert np.array_equal(cols.mu, [1.0, 10.0]) and cols.face == (W.FREESLIP,) * 6
    lay = W.viscosity_layers(n)
    assert np.array_equal(lay.cell_id, np.floor(4 * z).astype(np.uint8))
    assert np.array_equal(lay.mu, [1.0, 10.0, 100.0, 1000.0]) and lay.face == (W.FREESLIP,) * 6
    # the forcing of both: f = (0, 0, -cos(2 pi x) cos(2 pi y) sin(pi z)), at a few nodes
    for p in (cols, lay):
        f = p.nodal_forcing()
        nn = n + 1
        for (i, j, k), want in (((0, 0, 8), -1.0), ((8, 0, 8), 1.0), ((4, 0, 8), 0.0), ((0, 0, 0), 0.0),
                                ((8, 8, 4), -np.sin(np.pi / 4))):
            assert abs(f[2, i + nn * (j + nn * k)] - want) <= 1e-15
        assert np.all(f[0] == 0) and np.all(f[1] == 0)


def test_level_set_sphere_cuts_the_coarse_cells():
    p = W.level_set_sphere(32, 4)
    assert set(np.unique(p.cell_id)) == {0, 1}
    assert not _resolved_on(p.cell_id, 32, 4)  # not aligned with the coarse grid
    assert np.array_equal(p.mu, [1.0, 1e3]) and p.face == (W.DIRICHLET,) * 6


def test_random_vector_recipe():
    v = W.random_vector(8, 5)
    assert v.shape == (4, 9 ** 3) and v.dtype == np.float64
    assert np.array_equal(v, W.random_vector(8, 5))
    assert -1.0 <= v.min() < -0.9 and 0.9 < v.max() <= 1.0
    assert not np.array_equal(v, W.random_vector(8, 6))
