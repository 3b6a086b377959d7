"""The seeded input generators shared by the CUDA path's tests and benchmark and by the oracle: the
same seed gives the same arrays, the element maps are consistent with the node lattice, and the
derived meshes (tetrahedra, Q2) sit on the Q1 box they are built from, and the coefficient fields
follow their stated recipes."""
import numpy as np
import pytest

from paper_2308_09839_gb300 import inputs


@pytest.mark.parametrize("make", [
    lambda s: inputs.laplace_box(5, ny=4, nz=3, jitter=0.2, seed=s),
    lambda s: inputs.elasticity_box(4, jitter=0.1, seed=s),
    lambda s: inputs.vector_laplace_box(3, ny=5, nz=2, graded=0.3, seed=s),
    lambda s: inputs.tet_box("elasticity", 3, jitter=0.1, seed=s),
    lambda s: inputs.q2_box("laplace", 2, ny=3, nz=2, jitter=0.1, curve=0.05, seed=s),
])
def test_generators_are_seeded(make):
    a, b, c = make(3), make(3), make(4)
    for f in ("coords", "mat", "dirichlet"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert np.array_equal(a.cell_array(), b.cell_array())
    assert not np.array_equal(a.mat, c.mat)
    assert np.array_equal(a.x(1), b.x(1)) and np.array_equal(a.b(2), b.b(2))
    assert np.all(a.x(1)[a.dirichlet_dofs()] == 0.0)


def test_q2_lattice_sits_on_the_q1_box():
    n, ny, nz = 3, 2, 4
    p = inputs.q2_box("laplace", n, ny=ny, nz=nz, jitter=0.15, seed=5)
    V = inputs.box_coords(n, ny, nz, 0.15, 5)
    hexes = inputs.box_cells(n, ny, nz)
    corner = [0, 2, 6, 8, 18, 20, 24, 26]  # Q2 nodes at the Q1 corners, in the Q1 corner order
    assert np.array_equal(p.coords[p.cells[:, corner]], V[hexes])
    # straight edges: an edge midpoint is the mean of its two vertices
    mid = p.coords[p.cells[:, 1]]
    assert np.allclose(mid, 0.5 * (p.coords[p.cells[:, 0]] + p.coords[p.cells[:, 2]]), atol=1e-15)
    # neighbouring elements share the face nodes
    e0, e1 = 0, 1  # x-neighbours
    assert np.array_equal(p.cells[e0].reshape(3, 3, 3)[:, :, 2], p.cells[e1].reshape(3, 3, 3)[:, :, 0])
    assert p.n_nodes == (2 * n + 1) * (2 * ny + 1) * (2 * nz + 1)
    assert p.dirichlet.sum() == (2 * n + 1) * (2 * ny + 1)


def test_tet_cells_split_each_hexahedron():
    n, ny, nz = 2, 3, 2
    p = inputs.tet_box("laplace", n, ny=ny, nz=nz, seed=6)
    hexes = inputs.box_cells(n, ny, nz)
    tets = p.cells.reshape(-1, 6, 4)
    for e in range(hexes.shape[0]):
        assert set(np.unique(tets[e])) == set(hexes[e])  # the 6 tetrahedra use the 8 corners
        assert np.all(tets[e][:, 0] == hexes[e][0]) and np.all(tets[e][:, 3] == hexes[e][7])
    assert np.array_equal(p.mat, np.repeat(inputs.laplace_box(n, ny=ny, nz=nz, seed=6, sigma=0.5,
                                                              layered=True).mat, 6))


def test_renumber_is_a_relabelling():
    p = inputs.laplace_box(3, ny=2, nz=4, jitter=0.2, seed=7)
    cells = p.cell_array()
    coords, new_cells, dirichlet, node_perm, elem_perm = inputs.renumber(p.coords, cells, p.dirichlet, seed=8)
    assert np.array_equal(np.sort(node_perm), np.arange(p.n_nodes))
    assert np.array_equal(coords[new_cells], p.coords[cells[elem_perm]])
    assert np.array_equal(dirichlet[node_perm], p.dirichlet)


def test_coefficient_recipes():
    """The coefficient fields follow their stated recipes: lognormal cells with log-sd sigma; eight
    equal z-slabs, each with one multiplier 10^s, s in [-1, 1]; the Gaussian random field has mean 0,
    standard deviation sigma, and the correlation of white noise smoothed by a Gaussian of c cells,
    exp(-d^2 / (4 c^2)) at lag d (estimated on a periodic 64^3 box, which biases it slightly low)."""
    import math
    lk = np.log(inputs.lognormal_cells(200000, 0.5, seed=3))
    assert abs(lk.mean()) < 0.01 and abs(lk.std() - 0.5) < 0.01
    m = inputs.layer_multiplier(6, 5, 16, 8, seed=4).reshape(16, 5, 6)
    s = np.log10(m[:, 0, 0])
    assert np.all(np.abs(s) <= 1.0)
    assert np.all(m == m[:, :1, :1])  # constant within each z-plane
    assert np.all(s[0::2] == s[1::2]) and len(set(s[0::2])) == 8  # 8 slabs of 2 planes
    f = inputs.gaussian_random_field(64, 64, 64, 4.0, 1.5, seed=0).reshape(64, 64, 64)
    assert abs(f.mean()) < 1e-12 and abs(f.std() - 1.5) < 1e-12
    for d, tol in ((2, 0.02), (4, 0.05), (8, 0.1)):
        c = np.mean([np.mean(f * np.roll(f, d, axis=a)) for a in range(3)]) / f.var()
        assert abs(c - math.exp(-d * d / (4 * 16.0))) < tol, (d, c)
