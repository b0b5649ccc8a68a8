"""Pins of the oracle's sedimentation."""
import numpy as np

from oracle import sedi
from workloads import grid_global


def test_sutherland_reference_point():
    # Sutherland's formula is normalised to 1.8325e-5 Pa s at 296.16 K
    assert abs(sedi.viscosity(296.16) - 1.8325e-5) < 1e-12
    assert 1.78e-5 < sedi.viscosity(288.15) < 1.80e-5


def test_textbook_settling_velocity_order_of_magnitude():
    # a 2 micrometre-diameter unit-density particle at sea level settles at about 1.3e-4 m/s
    v = sedi.settling_velocity(101325.0, 293.15, 1e-6, 1000.0)
    assert 1.2e-4 < v < 1.45e-4


def test_stokes_limit_and_slip_correction_limits():
    p, T, rho_p = 101325.0, 288.15, 2000.0
    # large particles: Kn -> 0, the correction vanishes, v = 2 r^2 (rho_p - rho) g / (9 eta)
    r = 50e-6
    rho = p / (sedi.R_D * T)
    stokes = 2 * r * r * (rho_p - rho) * sedi.G / (9 * sedi.viscosity(T))
    assert abs(sedi.settling_velocity(p, T, r, rho_p) / stokes - 1) < 3e-3
    # velocity grows as r^2 times the correction: doubling a small r gives between 2x and 4x
    v1 = sedi.settling_velocity(p, T, 0.05e-6, rho_p)
    v2 = sedi.settling_velocity(p, T, 0.1e-6, rho_p)
    assert 2.0 < v2 / v1 < 4.0
    # thin air: the slip correction (Kn large) makes the fall faster than Stokes
    assert sedi.settling_velocity(1000.0, 220.0, 1e-6, rho_p) > 5 * sedi.settling_velocity(1e5, 220.0, 1e-6, rho_p)


def test_sediment_steps_increase_pressure_by_rho_g_v_dt():
    grid = grid_global(12, 7, 5, 1e5, 1e4)
    T = np.full((5, 7, 12), 250.0)
    st = {"lon": np.array([10.0, 200.0]), "lat": np.array([0.0, 30.0]), "p": np.array([5e4, 3e4])}
    r, rho_p = np.full(2, 5e-6), np.full(2, 2500.0)
    p1 = sedi.sediment(grid, T, 0.0, T, 3600.0, st, r, rho_p, 0.0, 60.0, 1)
    vs = sedi.settling_velocity(st["p"], 250.0, r, rho_p)
    np.testing.assert_allclose(p1 - st["p"], st["p"] / (sedi.R_D * 250.0) * sedi.G * vs * 60.0, rtol=1e-12)
    assert np.all(p1 > st["p"])
