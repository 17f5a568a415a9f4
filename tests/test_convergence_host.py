"""Host logic of the mesh-refinement study (no GPU): the nested O-mesh family and the observed-order
estimate."""
import numpy as np
import pytest

from paper_2501_00923_gb300 import convergence as C


def test_nested_meshes_nest_exactly():
    """Every node of a level is a node of the next (angular and radial counts double, the radial
    stretching ratio goes to its square root)."""
    meshes = C._nested_meshes([(16, 8), (32, 16), (64, 32)])
    for a, b in zip(meshes[:-1], meshes[1:]):
        assert np.abs(b.nodes[::2, ::2] - a.nodes).max() < 1e-13
        assert b.ni == 2 * a.ni and b.nj == 2 * a.nj


def test_nested_meshes_reject_non_doubling_sizes():
    with pytest.raises(ValueError):
        C._nested_meshes([(16, 8), (32, 12)])


@pytest.mark.parametrize("p", [1.0, 1.25, 2.0])
def test_observed_order_recovers_a_power_law(p):
    """J_h = J* + c h^p on halved spacings: the estimate returns p and the Richardson value J*."""
    J = [0.94 + 0.3 * (0.5 ** k) ** p for k in range(4)]
    order, Jinf = C._observed(J)
    assert abs(order - p) < 1e-9
    assert abs(Jinf - 0.94) < 1e-12


def test_observed_order_needs_three_monotone_levels():
    assert C._observed([1.0, 0.9]) == (None, None)
    assert C._observed([1.0, 0.9, 0.95]) == (None, None)     # oscillating differences
