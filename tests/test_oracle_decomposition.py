"""Pins of the oracle's decomposition (Def. 2.3, 3.2, 2.7): a hand count and
the partition-of-unity identity used in the stable decomposition (Lemma 3.3)."""
import json
import os

import numpy as np
import pytest

from oracle import decomposition as D
from paper_2406_06283_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "decomp_h8_p2_ov1.json")


def test_hand_count_h8_p2_ov1():
    g = json.load(open(GOLDEN))
    m = W.square_mesh(g["cells"])
    e2s = W.box_partition(m, g["parts"])
    subs, mu = D.decompose(m.xyz, m.elems, m.is_boundary, e2s, 4, g["overlap"])
    assert [s.elems.size for s in subs] == g["n_elems_overlapping"]
    assert [s.ovdof.size for s in subs] == g["n_ovdof"]
    assert [s.dof.size for s in subs] == g["n_dof"]
    dofs = W.dof_numbering(m)
    node = lambda i, j: j * (g["cells"] + 1) + i  # noqa: E731
    assert mu[dofs[node(4, 4)]] == g["mu_at_node_4_4"]
    assert mu[dofs[node(4, 1)]] == g["mu_at_node_4_1"]
    assert mu[dofs[node(1, 1)]] == g["mu_at_node_1_1"]


@pytest.mark.parametrize("cells,parts,ov", [(16, 2, 1), (24, 3, 2), (20, 3, 1), (32, 4, 2)])
def test_partition_of_unity_identity(cells, parts, ov):
    # sum_i E_i Xi_i R_i = I: every dof is internal to some subdomain and the
    # 1/mu weights of the subdomains containing it add up to one.
    m = W.square_mesh(cells)
    e2s = W.box_partition(m, parts)
    subs, mu = D.decompose(m.xyz, m.elems, m.is_boundary, e2s, parts * parts, ov)
    n = m.n_dofs
    acc = np.zeros(n)
    for s in subs:
        assert np.all(np.isin(s.dof, s.ovdof))
        w = D.pou_weights(s, mu)
        acc[s.ovdof] += w
    np.testing.assert_allclose(acc, 1.0, rtol=1e-15)
    assert mu.min() >= 1


def test_extension_is_monotone_and_layered():
    m = W.square_mesh(16)
    e2s = W.box_partition(m, 4)
    base = e2s == 5
    one = D.extend_by_layers(m.elems, m.is_boundary, base, 1)
    two = D.extend_by_layers(m.elems, m.is_boundary, base, 2)
    again = D.extend_by_layers(m.elems, m.is_boundary, one, 1)
    assert np.all(one[base]) and np.all(two[one])
    np.testing.assert_array_equal(two, again)


def test_lambda_multiplicity():
    m = W.square_mesh(16)
    e2s = W.box_partition(m, 4)
    subs, _ = D.decompose(m.xyz, m.elems, m.is_boundary, e2s, 16, 1)
    assert D.multiplicity_lambda(m.elems, subs, m.n_elems) == 4


def test_3d_partition_of_unity():
    m = W.cube_mesh(6)
    e2s = W.box_partition(m, 2)
    subs, mu = D.decompose(m.xyz, m.elems, m.is_boundary, e2s, 8, 1)
    acc = np.zeros(m.n_dofs)
    for s in subs:
        acc[s.ovdof] += D.pou_weights(s, mu)
    np.testing.assert_allclose(acc, 1.0, rtol=1e-15)
