"""Plant known mistakes in the oracle (on the CPU) and check that the pins
catch each one.  The switch lives in the oracle's C source and is off
except inside this test."""
import pytest

import oracle
import _pins

# mutation -> what it plants
MUTATIONS = {
    1: "gradient uses 1/2 (f_i + f_j) instead of 1/2 (f_j - f_i)",
    2: "face conormal sign not oriented from a to b",
    3: "face tangent sign reversed",
    5: "one of the two sub-triangles dropped from the dual volume",
    6: "east and north gradient components swapped",
    7: "divergence: the node's own wind dropped from the edge average",
    8: "curl: tangent not negated for the edge's second node",
    9: "gradient normalised by a neighbour's dual volume",
    10: "triangle centroid not projected to the sphere",
    12: "equally spaced latitudes instead of the Gaussian rows",
    13: "rows start half a spacing east of longitude 0",
    14: "Laplacian: gradient components swapped before the divergence",
}


def _all_pins(m):
    return {
        "gauss_rows": _pins.pin_gaussian_rows(m),
        "longitudes": _pins.pin_longitudes(m),
        "grad_const": _pins.pin_grad_constant(m),
        "volume": _pins.pin_total_volume(m),
        "closed": _pins.pin_closed_tangent(m),
        "brute": _pins.pin_bruteforce(m),
        "conservation": _pins.pin_conservation(m),
        "grad_analytic": _pins.pin_grad_analytic(m, 0.1),
        "solid_body": _pins.pin_solid_body(m, 2e-3, 9e-3),
        "wind": _pins.pin_wind(m, 0.12),
        "lap_eigen": _pins.pin_lap_eigen(m, 5, 0.1),
    }


def test_pins_pass_without_mutation():
    m = oracle.build_mesh(16)
    res = _all_pins(m)
    assert all(ok for ok, _ in res.values()), res


@pytest.mark.parametrize("mut", sorted(MUTATIONS))
def test_planted_mistake_is_caught(mut):
    oracle.set_mutation(mut)
    try:
        m = oracle.build_mesh(16)
        res = _all_pins(m)
    finally:
        oracle.set_mutation(0)
    failed = [k for k, (ok, _) in res.items() if not ok]
    assert failed, f"mutation {mut} ({MUTATIONS[mut]}) passed every pin: {res}"
