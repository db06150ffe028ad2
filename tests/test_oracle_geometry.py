"""Oracle median-dual geometry pins."""
import numpy as np
import pytest

import _pins


@pytest.mark.parametrize("N", [16, 32, 64])
def test_dual_cells_tile_the_sphere(N, mesh_factory):
    m = mesh_factory(N)
    ok, msg = _pins.pin_total_volume(m)
    assert ok, msg
    assert np.all(m.vol > 0)


@pytest.mark.parametrize("N", [16, 32])
def test_dual_boundaries_are_closed(N, mesh_factory):
    ok, msg = _pins.pin_closed_tangent(mesh_factory(N))
    assert ok, msg


def test_edge_assembly_equals_direct_dual_cell_walk_o16(mesh_factory):
    ok, msg = _pins.pin_bruteforce(mesh_factory(16))
    assert ok, msg


def test_edge_assembly_equals_direct_walk_sampled_o32(mesh_factory):
    m = mesh_factory(32)
    nodes = list(range(0, 40)) + list(range(2600, 2650)) + list(range(m.V - 40, m.V))
    ok, msg = _pins.pin_bruteforce(m, nodes=nodes)
    assert ok, msg


def test_face_normal_points_from_first_to_second_node(mesh_factory):
    m = mesh_factory(32)
    xyz = np.stack([np.cos(m.lat) * np.cos(m.lon), np.cos(m.lat) * np.sin(m.lon), np.sin(m.lat)], 1)
    ab = xyz[m.edge[:, 1]] - xyz[m.edge[:, 0]]
    assert np.all(np.einsum("ij,ij->i", m.S, ab) > 0)
    # the face is short compared with the sphere: |S| < |T| + pi R / N
    assert np.all(np.linalg.norm(m.S, axis=1) > 0)
