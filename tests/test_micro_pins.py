"""Pins of the oracle's droplet microphysics (paper Sec. 2.1: the vapour mass-transfer equation, the
droplet heat balance, and the vapour-mass and energy sources), each against something other than the
oracle's own formulas: steam tables, the conduction limit of a sphere, scipy integration of the
equations in the paper's mass form, the psychrometric wet-bulb temperature, exact conservation and
the order of convergence."""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pins.json")))
PI = math.pi


def _grid(n=4, g=(0.0, 0.0, 0.0), **kw):
    return oracle.make_grid(n, g=g, **kw)


def _uniform(G, u=(0.0, 0.0, 0.0), Tf=290.0, rv=0.01):
    nc = oracle.ncell(G)
    U = np.tile(np.asarray(u, dtype=float), (nc, 1))
    return U, np.full(nc, float(Tf)), np.full(nc, float(rv))


def _one(d0, T0, v0=(0.0, 0.0, 0.0), x0=(0.3, 0.4, 0.6)):
    return (np.array(x0, dtype=float).reshape(3, 1), np.array(v0, dtype=float).reshape(3, 1), np.array([d0]),
            np.array([T0]))


def test_saturation_vapour_density_matches_tables():
    g = GOLD["saturation_vapour_density"]
    for T, rho in zip(g["T_K"], g["rho_g_per_m3"]):
        assert abs(oracle.rho_sat(T) * 1e3 - rho) <= g["rel_tol"] * rho, (T, oracle.rho_sat(T))
    # increasing with temperature
    Ts = np.linspace(260, 320, 61)
    assert np.all(np.diff([oracle.rho_sat(T) for T in Ts]) > 0)


def test_nusselt_conduction_limit_and_correlation():
    g = GOLD["ranz_marshall_nusselt"]
    M = oracle.make_micro(Pr=g["Pr"])
    for re, nu in g["cases"]:
        assert abs(oracle.nusselt(M, re) - nu) <= g["abs_tol"]


@pytest.mark.parametrize("sat", [1.3, 0.7])
@pytest.mark.parametrize("mult", [1.0, 3.0])
def test_d_squared_law_matches_the_mass_equation(sat, mult):
    """Isothermal droplet (no latent heat, T_p = T_f): the paper's dm/dt = 2 pi D_v d rho_sat (S_f - S_p)
    integrated by scipy in mass form matches the oracle's steps; n steps of dt equal one step of n dt."""
    from scipy.integrate import solve_ivp

    G = _grid(mult=mult)
    M = oracle.make_micro(L=0.0)
    Tf = 290.0
    rs = oracle.rho_sat(Tf)
    U, T, R = _uniform(G, Tf=Tf, rv=sat * rs)
    x, v, d, Tp = _one(20e-6, Tf)
    steps, dt = 50, 1e-3
    _, _, d1, T1, _, msrc, _ = oracle.micro_run(G, M, U, T, R, x, v, d, Tp, steps, dt)
    _, _, d2, _, _, _, _ = oracle.micro_run(G, M, U, T, R, x, v, d, Tp, 1, steps * dt)
    rho_p = 1000.0

    def rhs(t, y):
        m = y[0]
        dd = (6.0 * m / (rho_p * PI)) ** (1.0 / 3.0)
        return [2.0 * PI * M.D_v * dd * rs * (sat - 1.0)]

    m0 = rho_p * PI * 20e-6 ** 3 / 6.0
    sol = solve_ivp(rhs, (0.0, steps * dt), [m0], method="DOP853", rtol=1e-13, atol=1e-30)
    d_ode = (6.0 * sol.y[0, -1] / (rho_p * PI)) ** (1.0 / 3.0)
    assert abs(d1[0] - d_ode) <= 1e-11 * d_ode
    assert abs(d1[0] - d2[0]) <= 1e-13 * d_ode
    assert (d1[0] > 20e-6) == (sat > 1.0)
    assert T1[0] == Tf  # no latent heat, no temperature difference: T_p stays
    # the vapour the fluid gains is the mass the parcel lost (multiplicity included)
    dm_parcel = mult * rho_p * PI * (d1[0] ** 3 - 20e-6 ** 3) / 6.0
    assert abs(msrc.sum() + dm_parcel) <= 1e-12 * abs(dm_parcel)


@pytest.mark.parametrize("d0", [10e-6, 40e-6])
def test_temperature_relaxes_without_mass_transfer(d0):
    """D_v = 0, no slip: m C_p dT/dt = pi Nu kappa d (T_f - T) with Nu = 2, integrated by scipy."""
    from scipy.integrate import solve_ivp

    G = _grid()
    M = oracle.make_micro(D_v=0.0)
    U, T, R = _uniform(G, u=(0.2, -0.1, 0.05), Tf=290.0, rv=0.0)
    x, v, d, Tp = _one(d0, 300.0, v0=(0.2, -0.1, 0.05))
    steps, dt = 40, 2.5e-3
    _, v1, d1, T1, _, _, _ = oracle.micro_run(G, M, U, T, R, x, v, d, Tp, steps, dt)
    assert d1[0] == d0
    m = 1000.0 * PI * d0 ** 3 / 6.0
    sol = solve_ivp(lambda t, y: [PI * 2.0 * M.kappa_f * d0 * (290.0 - y[0]) / (m * M.cp_p)], (0.0, steps * dt),
                    [300.0], method="DOP853", rtol=1e-13, atol=1e-12)
    assert abs(T1[0] - sol.y[0, -1]) <= 1e-10 * 10.0


def test_evaporating_droplet_reaches_the_wet_bulb_temperature():
    """A droplet in air at 20 degC and 50 % relative humidity, no slip: evaporation cools it below the air
    until conduction balances the latent heat (the latent heat enters the droplet's heat balance with the
    sign that cools an evaporating droplet)."""
    g = GOLD["wet_bulb_20C_50pct"]
    G = _grid()
    M = oracle.make_micro()
    Ta = g["T_air_K"]
    U, T, R = _uniform(G, Tf=Ta, rv=g["relative_humidity"] * oracle.rho_sat(Ta))
    x, v, d, Tp = _one(200e-6, Ta)
    _, _, d1, T1, _, _, _ = oracle.micro_run(G, M, U, T, R, x, v, d, Tp, 6000, 1e-3)
    Tw = T1[0]
    assert Tw < Ta - 5.0
    assert abs(Tw - g["T_wet_bulb_K"]) <= g["abs_tol_K"], Tw
    # steady balance at Nu = 2: kappa (T_a - T_w) = L D_v (rho_sat(T_w) - rho_v)
    lhs = M.kappa_f * (Ta - Tw)
    rhs = M.L * M.D_v * (oracle.rho_sat(Tw) - g["relative_humidity"] * oracle.rho_sat(Ta))
    assert abs(lhs - rhs) <= 2e-3 * lhs
    assert d1[0] < 200e-6


def test_coupled_mass_and_heat_converge_to_the_equations():
    """Mass and heat transfer together (latent heat on), over a few thermal times of the droplet: the
    step converges to the coupled equations of Sec. 2.1 (integrated by scipy) at first order or better,
    and stays stable for steps longer than the thermal time."""
    from scipy.integrate import solve_ivp

    G = _grid()
    M = oracle.make_micro()
    Tf = 285.0
    rv = 1.03 * oracle.rho_sat(Tf)
    U, T, R = _uniform(G, Tf=Tf, rv=rv)
    d0, T0, Tend = 8e-6, 280.0, 3e-3
    rho_p = 1000.0

    def rhs(t, y):
        m, Tp = y
        dd = (6.0 * max(m, 1e-30) / (rho_p * PI)) ** (1.0 / 3.0)
        mdot = 2.0 * PI * M.D_v * dd * (rv - oracle.rho_sat(Tp))
        Tdot = (PI * 2.0 * M.kappa_f * dd * (Tf - Tp) + M.L * mdot) / (m * M.cp_p)
        return [mdot, Tdot]

    m0 = rho_p * PI * d0 ** 3 / 6.0
    sol = solve_ivp(rhs, (0.0, Tend), [m0, T0], method="Radau", rtol=1e-13, atol=[1e-27, 1e-13])
    d_ref = (6.0 * sol.y[0, -1] / (rho_p * PI)) ** (1.0 / 3.0)
    T_ref = sol.y[1, -1]
    errs = []
    for steps in (4, 8, 16, 32):
        x, v, d, Tp = _one(d0, T0)
        _, _, d1, T1, _, _, _ = oracle.micro_run(G, M, U, T, R, x, v, d, Tp, steps, Tend / steps)
        errs.append((abs(d1[0] - d_ref) / d_ref, abs(T1[0] - T_ref)))
    errs = np.array(errs)
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > 1.8), ratios
    assert errs[-1, 0] < 1e-5 and errs[-1, 1] < 1e-4
    # steps of 3 and 30 thermal times land near the quasi-steady temperature instead of oscillating
    sol = solve_ivp(rhs, (0.0, 0.03), [m0, T0], method="Radau", rtol=1e-12, atol=[1e-27, 1e-12])
    for steps, tol in ((1, 1.0), (10, 0.05)):
        x, v, d, Tp = _one(d0, T0)
        _, _, d1, T1, _, _, _ = oracle.micro_run(G, M, U, T, R, x, v, d, Tp, steps, 0.03 / steps)
        assert abs(T1[0] - sol.y[1, -1]) < tol and Tf < T1[0] < Tf + 1.0


def _random_case(n=2000, N=8, seed=5):
    from paper_2603_26691_gb300 import inputs

    G = oracle.make_grid(N, mult=2.0)
    U = inputs.random_fourier(N, seed=seed).reshape(-1, 3)
    x, y, z = inputs.cell_centres(N)
    Tf = (285.0 + 3.0 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * z)).reshape(-1)
    rv = np.array([oracle.rho_sat(t) for t in Tf]) * (1.0 + 0.05 * np.cos(2 * np.pi * y).reshape(-1))
    pos, vel, d, _ = inputs.particles(seed, 0, n, vmax=0.3)
    Tp = 283.0 + 4.0 * np.random.default_rng(seed).random(n)
    return G, U, Tf, rv, pos, vel, d, Tp


def test_water_energy_and_momentum_are_conserved():
    G, U, Tf, rv, pos, vel, d, Tp = _random_case()
    M = oracle.make_micro()
    dt, steps = 1e-3, 30
    gvec = np.array(G.g[:])
    mass = lambda dd: np.array([oracle.mass(G, x) for x in dd])  # noqa: E731
    m0 = mass(d)
    W0, E0, P0 = m0.sum(), (M.cp_p * m0 * Tp).sum(), (m0 * vel).sum(axis=1)
    grav = np.zeros(3)
    src = np.zeros((3, oracle.ncell(G)))
    ms = np.zeros(oracle.ncell(G))
    es = np.zeros(oracle.ncell(G))
    for _ in range(steps):
        grav += mass(d).sum() * gvec * dt
        pos, vel, d, Tp, s1, m1, e1 = oracle.micro_run(G, M, U, Tf, rv, pos, vel, d, Tp, 1, dt)
        src += s1
        ms += m1
        es += e1
    m = mass(d)
    assert abs(m.sum() + ms.sum() - W0) <= 1e-12 * W0
    assert abs((M.cp_p * m * Tp).sum() + es.sum() - E0) <= 1e-12 * E0
    P = (m * vel).sum(axis=1)
    scale = np.abs(src).sum() + np.abs(grav).max()
    assert np.abs(P - P0 - grav + src.sum(axis=1)).max() <= 1e-12 * scale
    # droplets both grew and shrank, and the fluid gained and lost vapour
    assert (ms > 0).any() and (ms < 0).any()


def test_without_transfer_it_is_the_plain_step():
    """No vapour diffusion and droplets at the fluid temperature everywhere: no mass or heat moves, and the
    motion and momentum source are those of the plain step."""
    G, U, Tf, rv, pos, vel, d, Tp = _random_case(n=500)
    Tf = np.full_like(Tf, 285.0)
    Tp = np.full_like(Tp, 285.0)
    M = oracle.make_micro(D_v=0.0)
    p1, v1, d1, T1, s1, m1, e1 = oracle.micro_run(G, M, U, Tf, rv, pos, vel, d, Tp, 12, 1e-3)
    p2, v2, s2, _ = oracle.run(G, U, pos, vel, d, 12, 1e-3)
    assert np.array_equal(d1, d) and np.abs(T1 - 285.0).max() <= 1e-12 * 285.0
    assert np.array_equal(p1, p2) and np.array_equal(v1, v2)
    assert np.abs(s1 - s2).max() <= 1e-13 * np.abs(s2).max()
    assert not m1.any()
    # the temperature moves only by the rounding of the gathered constant temperature field
    assert np.abs(e1).max() <= 1e-12 * M.cp_p * 285.0 * max(oracle.mass(G, x) for x in d)


def test_evaporation_stops_at_the_minimum_diameter():
    G = _grid()
    M = oracle.make_micro(L=0.0, d_min=1e-7)
    U, T, R = _uniform(G, Tf=300.0, rv=0.0)
    x, v, d, Tp = _one(3e-6, 300.0)
    _, _, d1, _, _, msrc, _ = oracle.micro_run(G, M, U, T, R, x, v, d, Tp, 200, 1e-3)
    assert d1[0] == 1e-7
    m0 = 1000.0 * PI * 3e-6 ** 3 / 6.0
    m1 = 1000.0 * PI * 1e-21 / 6.0
    assert abs(msrc.sum() - (m0 - m1)) <= 1e-12 * m0
