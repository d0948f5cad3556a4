"""Mutation checks of the oracle's observables: each test plants one plausible
mistake in a copy of oracle/sc_oracle.c (compiled into a temporary folder; the
built oracle is untouched) and requires the hand-built pins of
tests/test_oracle_diag.py to catch it. The mistakes are the ones a restatement
of Sec. III B / III C could make: dropping the linear interpolation of x_I,
interpolating from the wrong plane, taking any sign change or the last crossing,
ignoring the liquid base above a wall, counting rho^r >= rho^b, or a wrong
volume-to-radius formula."""
import os

import pytest

import test_oracle_diag as pins

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "sc_oracle.c")

INTERP = "d->interface_z = z + phi[z] / (phi[z] - phi[z + 1]);"
MUTANTS = {
    "no_interpolation": (INTERP, "d->interface_z = z;"),
    "weight_from_the_upper_plane": (INTERP, "d->interface_z = z + phi[z + 1] / (phi[z + 1] - phi[z]);"),
    "interpolated_from_the_lower_neighbour": (INTERP, "d->interface_z = z + phi[z] / (phi[z] - phi[z - 1 < 0 ? 0 : z - 1]);"),
    "offset_by_the_wrong_end": (INTERP, "d->interface_z = z + 1 - phi[z] / (phi[z] - phi[z + 1]);"),
    "any_sign_change": ("if (phi[z] > 0.0 && phi[z + 1] <= 0.0) {", "if ((phi[z] > 0.0) != (phi[z + 1] > 0.0)) {"),
    "last_crossing": ("      d->interface_z = z + phi[z] / (phi[z] - phi[z + 1]);\n      break;",
                      "      d->interface_z = z + phi[z] / (phi[z] - phi[z + 1]);"),
    "no_liquid_base": ("int z0 = p->wall_thickness > 0 ? p->wall_z0 + p->wall_thickness : 0;", "int z0 = 0;"),
    "ties_counted": ("if (rr > rb) ++cnt;", "if (rr >= rb) ++cnt;"),
    "radius_formula": ("d->radius = cbrt(3.0 * (double)cnt / (4.0 * M_PI));",
                       "d->radius = sqrt((double)cnt / M_PI);"),
}


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(oracle_mod, source, tmp_path, name):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, f"mutation site of {name} not found exactly once"
    lib = oracle_mod.compile_variant(source.replace(old, new), str(tmp_path), name)
    caught = bool(pins.check_interface_cases(oracle_mod, library=lib))
    for V in (317, 1000):
        caught = caught or not pins.check_radius(oracle_mod, library=lib, V=V)[0]
    assert caught, f"the pins do not catch the mutation {name}"


def test_unmutated_copy_passes(oracle_mod, source, tmp_path):
    """The harness itself: the same source, compiled the same way, passes every pin."""
    lib = oracle_mod.compile_variant(source, str(tmp_path), "same")
    assert pins.check_interface_cases(oracle_mod, library=lib) == []
    assert pins.check_radius(oracle_mod, library=lib)[0]
