"""Pins of the Sedov-Taylor similarity solution that the long-run GPU test compares
against: values published for it, and properties of the exact solution."""
import pytest

from _sedov import similarity


def test_taylor_constant_for_air():
    """gamma = 1.4: R = 1.033 (E t^2 / rho0)^(1/5) (Taylor 1950)."""
    assert similarity(1.4)["xi0"] == pytest.approx(1.033, abs=5e-4)


def test_monatomic_constant_and_energy_split():
    """gamma = 5/3: xi0 = 1.1517 (alpha = 0.4936), and the blast holds about 28 % of
    its energy as kinetic and 72 % as thermal energy."""
    s = similarity(5.0 / 3.0)
    assert s["xi0"] == pytest.approx(1.1517, abs=2e-4)
    assert s["e_kin_frac"] == pytest.approx(0.28, abs=0.005)


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_centre_and_shock_limits(gamma):
    """Near the centre the gas moves homologously with v = r / (gamma t), i.e.
    F = xi / gamma, the pressure stays finite and the density vanishes; at the shock
    the profiles take the strong-shock jump values."""
    s = similarity(gamma)
    for x in (1e-2, 3e-3):
        assert s["F"](x) == pytest.approx(x / gamma, rel=1e-3)
        assert s["G"](x) < 1e-6
    assert s["P"](1e-3) == pytest.approx(s["P"](1e-2), rel=1e-3)
    assert s["G"](1.0) == pytest.approx((gamma + 1) / (gamma - 1), rel=1e-12)
    # the density falls monotonically from the shock inwards
    xs = [1.0, 0.95, 0.9, 0.8, 0.6, 0.4]
    g = [s["G"](x) for x in xs]
    assert all(a > b for a, b in zip(g, g[1:]))
