"""Pins of the oracle's physics variants: the nearest-grid-point gather and semi-implicit Euler
integrator of Sec. 2.5, the Schiller-Naumann drag correlation cited in Sec. 2.1, and the
cloud-in-cell deposit (the transpose of the trilinear gather).  Each is checked against what the
mathematics or the physics fixes independently of the oracle's own formulas: closed forms of the
discrete recursion, an accurately integrated ODE written in the drag-force form, a force balance
at terminal velocity, the transpose identity with the pinned trilinear gather, and the momentum
budget of every combination."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2603_26691_gb300 import inputs

RHO_P, MU, G0 = 1000.0, 1.8e-5, np.array([0.0, 0.0, -9.81])


def _tau(d):
    return RHO_P * d * d / (18.0 * MU)


def _cd(re):
    """The Schiller-Naumann drag coefficient in its published drag-coefficient form."""
    return 24.0 / re * (1.0 + 0.15 * re ** 0.687) if re <= 1000.0 else 0.44


def _drag_accel(rho_f, d, rel):
    """Drag force per unit mass, 1/2 rho_f C_D (pi d^2/4) |rel| rel / (rho_p pi d^3/6)."""
    r = np.linalg.norm(rel)
    if r == 0.0:
        return np.zeros(3)
    re = rho_f * r * d / MU
    return 0.75 * rho_f * _cd(re) * r * rel / (RHO_P * d)


# ---- nearest grid point ----------------------------------------------------------------------

def test_ngp_gather_is_the_containing_cell_value_of_taylor_green():
    N = 8
    G = oracle.make_grid(N, gather="ngp")
    U = inputs.taylor_green(N)
    rng = np.random.default_rng(3)
    for x in rng.random((200, 3)):
        c = np.floor(x * N) + 0.5  # containing cell's centre, in cell units
        xc = c / N
        want = np.array([np.sin(2 * np.pi * xc[0]) * np.cos(2 * np.pi * xc[1]) * np.cos(2 * np.pi * xc[2]),
                         -np.cos(2 * np.pi * xc[0]) * np.sin(2 * np.pi * xc[1]) * np.cos(2 * np.pi * xc[2]),
                         0.0])
        assert np.abs(oracle.gather(G, U, x) - want).max() <= 1e-14


def test_ngp_is_piecewise_constant_and_jumps_at_faces():
    N = 6
    G = oracle.make_grid(N, gather="ngp")
    U = np.random.default_rng(4).normal(size=(N, N, N, 3))
    h = 1.0 / N
    y, z = 2.3 * h, 4.7 * h
    lo = oracle.gather(G, U, [3 * h - 1e-12, y, z])
    hi = oracle.gather(G, U, [3 * h + 1e-12, y, z])
    assert np.array_equal(lo, U[4, 2, 2]) and np.array_equal(hi, U[4, 2, 3])
    assert np.array_equal(oracle.gather(G, U, [3.1 * h, y, z]), oracle.gather(G, U, [3.9 * h, y, z]))


# ---- semi-implicit Euler ---------------------------------------------------------------------

def _uniform_run(G, n, dt, d, v0, u, x0=(0.5, 0.5, 0.5)):
    U = np.tile(np.asarray(u, float), (int(np.prod(G.n)), 1))
    pos = np.array(x0, float).reshape(3, 1)
    vel = np.asarray(v0, float).reshape(3, 1)
    p, v, _, _ = oracle.run(G, U, pos, vel, np.array([d]), n, dt)
    return p[:, 0], v[:, 0]


def test_semi_implicit_euler_matches_the_closed_form_of_its_recursion():
    # in a uniform flow v' = (v + dt (a u + g)) / (1 + a dt) is an affine map with fixed point
    # w = u + g / a; v_n = w + (v0 - w) r^n with r = 1 / (1 + a dt), and x_n = x0 + dt sum v_k
    G = oracle.make_grid(4, L=(1e3, 1e3, 1e3), integrator="semi_implicit")
    d, dt, n = 40e-6, 2e-3, 37
    a = 1.0 / _tau(d)
    u = np.array([0.3, -0.2, 0.1])
    v0 = np.array([1.0, 0.5, -2.0])
    w = u + G0 / a
    r = 1.0 / (1.0 + a * dt)
    x, v = _uniform_run(G, n, dt, d, v0, u, x0=(500.0, 500.0, 500.0))
    assert np.abs(v - (w + (v0 - w) * r ** n)).max() <= 1e-12 * np.abs(v0).max()
    xs = 500.0 + n * dt * w + dt * (v0 - w) * r * (1 - r ** n) / (1 - r)
    assert np.abs(x - xs).max() <= 1e-12 * 500.0


def test_semi_implicit_euler_keeps_terminal_velocity_exactly():
    G = oracle.make_grid(4, integrator="semi_implicit", g=(0.0, 0.0, -9.81))
    d, dt = 20e-6, 5e-4
    u = np.array([0.0, 0.0, 0.0])
    w = u + G0 * _tau(d)
    _, v = _uniform_run(G, 50, dt, d, w, u)
    assert np.abs(v - w).max() <= 1e-15


@pytest.mark.parametrize("integrator", ["semi_implicit", "exponential"])
def test_first_order_convergence_with_schiller_naumann_drag(integrator):
    # a 100 um droplet shot at 2 m/s through still air settles; Re starts near 13. Reference: the
    # ODE dv/dt = (drag force)/m + g written in the drag-coefficient form, integrated by RK4 with a
    # step far below the schemes' (its error is negligible at this step)
    G = oracle.make_grid(4, L=(1e3, 1e3, 1e3), integrator=integrator, drag="schiller_naumann", rho_f=1.2)
    d, T = 100e-6, 0.02
    v0 = np.array([2.0, 0.0, 0.5])
    u = np.zeros(3)

    def rhs(v):
        return _drag_accel(1.2, d, u - v) + G0

    h = T / 20000
    v = v0.copy()
    for _ in range(20000):
        k1 = rhs(v)
        k2 = rhs(v + 0.5 * h * k1)
        k3 = rhs(v + 0.5 * h * k2)
        k4 = rhs(v + h * k3)
        v = v + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    errs = []
    for n in (40, 80, 160, 320):
        _, vn = _uniform_run(G, n, T / n, d, v0, u, x0=(500.0, 500.0, 500.0))
        errs.append(np.abs(vn - v).max())
    ratios = [errs[i + 1] / errs[i] for i in range(len(errs) - 1)]
    assert all(0.4 <= q <= 0.6 for q in ratios), (errs, ratios)


# ---- Schiller-Naumann ------------------------------------------------------------------------

def test_schiller_naumann_reduces_to_stokes_at_vanishing_reynolds_number():
    Gs = oracle.make_grid(8, drag="stokes")
    Gn = oracle.make_grid(8, drag="schiller_naumann", rho_f=0.0)
    U = inputs.taylor_green(8)
    pos, vel, d, _ = inputs.particles(5, 0, 64, vmax=0.5)
    a = oracle.run(Gs, U, pos, vel, d, 5, 1e-3)
    b = oracle.run(Gn, U, pos, vel, d, 5, 1e-3)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    Gt = oracle.make_grid(8, drag="schiller_naumann")
    assert abs(oracle.drag_factor(Gt, 1e-9) - 1.0) <= 1e-6


def test_schiller_naumann_terminal_velocity_balances_weight():
    # at terminal velocity in still air the drag force 1/2 rho_f C_D (pi d^2/4) v^2 equals the
    # weight m g: the scheme's fixed point, reached by stepping, satisfies the force balance
    for d in (100e-6, 300e-6, 1e-3):
        G = oracle.make_grid(4, L=(1e3, 1e3, 1e3), drag="schiller_naumann", rho_f=1.2)
        _, v = _uniform_run(G, 4000, 5e-3, d, np.zeros(3), np.zeros(3), x0=(500.0, 500.0, 500.0))
        vt = -v[2]
        re = 1.2 * vt * d / MU
        drag = 0.5 * 1.2 * _cd(re) * np.pi * d * d / 4 * vt * vt
        weight = RHO_P * np.pi * d ** 3 / 6 * 9.81
        assert abs(drag - weight) <= 1e-9 * weight, (d, re)
        assert abs(v[0]) + abs(v[1]) == 0.0
        # and it is below the Stokes terminal velocity (the correlation adds drag at Re > 0)
        assert vt < _tau(d) * 9.81


def test_schiller_naumann_newton_regime_and_continuity():
    G = oracle.make_grid(4, drag="schiller_naumann")
    # above Re = 1000 the drag coefficient is constant: f = C_D Re / 24 is linear in Re
    assert abs(oracle.drag_factor(G, 4000.0) / oracle.drag_factor(G, 2000.0) - 2.0) <= 1e-15
    assert abs(oracle.drag_factor(G, 2000.0) - 0.44 * 2000.0 / 24.0) <= 1e-12
    # the two branches meet at Re = 1000 to within the correlation's 0.3 % step
    lo, hi = oracle.drag_factor(G, 1000.0), oracle.drag_factor(G, 1000.0 * (1 + 1e-12))
    assert abs(hi / lo - 1.0) <= 4e-3
    # monotone in Re
    re = np.geomspace(1e-3, 1e5, 400)
    f = np.array([oracle.drag_factor(G, r) for r in re])
    assert np.all(np.diff(f) > 0.0)


# ---- cloud in cell ---------------------------------------------------------------------------

def test_cic_deposit_is_the_transpose_of_the_trilinear_gather():
    # <deposit(J at x), U> = J . gather(U, x) for every field U: the corner cells, weights and
    # periodic wrap of the deposit are those of the (pinned) trilinear gather
    G = oracle.make_grid((5, 4, 6), L=(1.0, 0.8, 1.2), deposit="cic")
    Gt = oracle.make_grid((5, 4, 6), L=(1.0, 0.8, 1.2))
    rng = np.random.default_rng(6)
    for _ in range(50):
        x = rng.random(3) * np.array([1.0, 0.8, 1.2])
        J = rng.normal(size=3)
        U = rng.normal(size=(6, 4, 5, 3))
        src = oracle.deposit(G, x, J)
        lhs = np.sum(src * U.reshape(-1, 3).T)
        rhs = J @ oracle.gather(Gt, U, x)
        assert abs(lhs - rhs) <= 1e-13 * (np.abs(J).sum() * np.abs(U).max())
        assert np.abs(src.sum(1) - J).max() <= 1e-15 * np.abs(J).max() * 8


def test_cic_deposit_special_positions():
    N = 4
    G = oracle.make_grid(N, deposit="cic")
    h = 1.0 / N
    J = np.array([1.0, -2.0, 3.0])
    c = lambda i, j, k: i + N * (j + N * k)
    # at a cell centre: everything into that cell
    src = oracle.deposit(G, [1.5 * h, 2.5 * h, 0.5 * h], J)
    assert np.array_equal(src[:, c(1, 2, 0)], J) and np.count_nonzero(src) == 3
    # on the face between cells 1 and 2 in x, centred in y and z: half into each
    src = oracle.deposit(G, [2.0 * h, 2.5 * h, 0.5 * h], J)
    assert np.array_equal(src[:, c(1, 2, 0)], J / 2) and np.array_equal(src[:, c(2, 2, 0)], J / 2)
    # next to x = 0 the stencil wraps to the last cell
    src = oracle.deposit(G, [0.25 * h, 2.5 * h, 0.5 * h], J)
    assert np.allclose(src[:, c(3, 2, 0)], J * 0.25, rtol=0, atol=1e-15)
    assert np.allclose(src[:, c(0, 2, 0)], J * 0.75, rtol=0, atol=1e-15)


# ---- every combination -----------------------------------------------------------------------

@pytest.mark.parametrize("gather,integrator,drag,deposit",
                         list(itertools.product(["trilinear", "ngp"], ["exponential", "semi_implicit"],
                                                ["stokes", "schiller_naumann"], ["cell", "cic"])))
def test_momentum_budget_of_every_physics_combination(gather, integrator, drag, deposit):
    # sum_p m (v(T) - v(0)) - (sum m) g T + sum_c J_c = 0 for any gather, integrator, drag and deposit
    N = 6
    G = oracle.make_grid(N, gather=gather, integrator=integrator, drag=drag, deposit=deposit)
    U = inputs.taylor_green(N)
    pos, vel, d, _ = inputs.particles(8, 0, 300, vmax=0.3)
    steps, dt = 7, 1e-3
    p, v, src, _ = oracle.run(G, U, pos, vel, d, steps, dt)
    m = np.array([oracle.mass(G, x) for x in d])
    dP = (m * (v - vel)).sum(1) - m.sum() * G0 * steps * dt
    scale = (m * np.abs(v - vel)).sum() + m.sum() * 9.81 * steps * dt
    assert np.abs(dP + src.sum(1)).max() <= 1e-12 * scale
    if deposit == "cell":
        # the containing-cell deposit only touches cells that held a particle at a step start
        assert np.count_nonzero(np.abs(src).sum(0)) <= min(N ** 3, 300 * steps)


def test_schiller_naumann_drag_coefficient_at_stored_values():
    import json
    import os

    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pins.json")))["schiller_naumann_cd"]
    G = oracle.make_grid(4, drag="schiller_naumann")
    for re, cd in golden["re_and_cd"]:
        assert abs(oracle.drag_factor(G, re) * 24.0 / re - cd) <= 1e-13 * cd, (re, cd)
