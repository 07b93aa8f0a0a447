"""Pins of the seeded input generator: SplitMix64 against its published
first outputs for seed 0, mesh counts, partition shapes."""
import numpy as np

from paper_2406_06283_gb300 import workloads as W


def test_splitmix64_reference_values():
    got = [int(x) for x in W.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_and_normal_ranges():
    u = W.uniform(W.stream_seed(1, 2), 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    z = W.normal(W.stream_seed(3), 100000)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02


def test_square_mesh_counts():
    m = W.square_mesh(64)
    assert m.n_nodes == 65 * 65 and m.n_elems == 2 * 64 * 64 and m.n_dofs == 3969
    assert W.square_mesh(256).n_dofs == 65025


def test_cube_mesh_counts():
    m = W.cube_mesh(4)
    assert m.n_elems == 6 * 64 and m.n_dofs == 27
    # Kuhn tets of one cube tile it: 6 tets of volume 1/6 each.
    P = m.xyz[m.elems]
    vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6
    np.testing.assert_allclose(vol.sum(), 1.0)


def test_box_partition_uneven():
    m = W.square_mesh(10)
    sub = W.box_partition(m, 3)
    counts = np.bincount(sub, minlength=9)
    assert counts.sum() == m.n_elems and counts.min() > 0


def test_config_shapes():
    p = W.config_c2()
    assert p.rhs.shape == (1, 65025) and p.n_sub == 64
    assert p.coeff.min() >= 1.0 and p.coeff.max() <= 100.0
    assert len(np.unique(p.coeff)) == 64
