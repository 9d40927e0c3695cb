"""Pins for the FP64 oracle: each test checks it against something other than
itself (textbook physics, an independent ODE solver, library routines, exact
rational arithmetic, conservation, finite differences)."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2603_26691_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pins.json")))


def _grid(o, n=8, **kw):
    return o.make_grid(n, **kw)


# --- integrator (Sec. 2.1, Eqs. 9-10 with Stokes drag and gravity) -------------------

@pytest.mark.parametrize("d", [5e-6, 2e-5, 8e-5])
@pytest.mark.parametrize("alpha", [1.0, 0.7])
def test_uniform_flow_matches_independent_ode_solution(oracle_mod, d, alpha):
    """Stokes drag written as the textbook force 3 pi mu d (u - v), integrated by DOP853."""
    from scipy.integrate import solve_ivp

    o = oracle_mod
    u = np.array([0.3, -0.2, 0.1])
    G = _grid(o, 16, alpha=alpha)
    U = inputs.uniform_field(16, u)
    x0 = np.array([0.31, 0.52, 0.77])
    v0 = np.array([0.9, -0.4, 0.25])
    dt, nsteps = 5e-4, 40
    m = 1000.0 * math.pi * d ** 3 / 6.0
    g = np.array([0.0, 0.0, -9.81])

    def rhs(t, y):
        v = y[3:]
        F = alpha * 3.0 * math.pi * 1.8e-5 * d * (u - v) + m * g
        return np.concatenate([v, F / m])

    T = dt * nsteps
    sol = solve_ivp(rhs, (0.0, T), np.concatenate([x0, v0]), method="DOP853", rtol=1e-13, atol=1e-15)
    pos, vel, _, _ = o.run(G, U, x0.reshape(3, 1), v0.reshape(3, 1), np.array([d]), nsteps, dt)
    xe = sol.y[:3, -1]
    ve = sol.y[3:, -1]
    dx = (pos[:, 0] - xe + 0.5) % 1.0 - 0.5  # minimum image in the unit box
    assert np.max(np.abs(dx)) < 1e-11
    assert np.max(np.abs(vel[:, 0] - ve)) < 1e-10 * (1.0 + np.max(np.abs(ve)))


def test_integrator_is_exact_for_frozen_flow(oracle_mod):
    """n steps of dt equal one step of n dt when the fluid velocity is frozen."""
    o = oracle_mod
    G = _grid(o, 16)
    up = np.array([0.3, -0.2, 0.1])
    for d in (3e-6, 2e-5, 1e-4):
        x, v = np.array([0.1, 0.2, 0.3]), np.array([1.0, -0.5, 0.2])
        xa, va = x.copy(), v.copy()
        for _ in range(25):
            xa, va = o.advance(G, d, up, 2e-4, xa, va)
        xb, vb = o.advance(G, d, up, 25 * 2e-4, x, v)
        assert np.max(np.abs(xa - xb)) < 1e-14
        assert np.max(np.abs(va - vb)) < 1e-13


def test_terminal_velocity_is_stokes_settling(oracle_mod):
    pin = GOLDEN["stokes_settling_20um"]
    o = oracle_mod
    G = _grid(o, 16)
    x, v = np.zeros(3), np.zeros(3)
    for _ in range(200):  # 200 ms >> tau = 1.23 ms
        x, v = o.advance(G, pin["d"], np.zeros(3), 1e-3, x, v)
    assert abs(v[2] + pin["v_settle"]) < 1e-12
    assert abs(v[0]) < 1e-15 and abs(v[1]) < 1e-15


# --- trilinear gather ------------------------------------------------------------------

def _trilinear_poly(x, y, z, c):
    return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * y * z + c[6] * x * z
            + c[7] * x * y * z)


def test_gather_reproduces_trilinear_functions(oracle_mod):
    """Trilinear interpolation is exact on span{1,x,y,z,xy,yz,xz,xyz} away from the seam."""
    o = oracle_mod
    n = (6, 7, 9)
    G = o.make_grid(n, L=(1.0, 2.0, 0.5))
    X, Y, Z = inputs.cell_centres(n, (1.0, 2.0, 0.5))
    rng = np.random.default_rng(0)
    coefs = rng.standard_normal((3, 8))
    U = np.stack([_trilinear_poly(X, Y, Z, coefs[q]) for q in range(3)], axis=-1)
    for _ in range(200):
        p = np.array([rng.uniform(0.5 / 6, 1.0 - 0.5 / 6), rng.uniform(1.0 / 7, 2.0 - 1.0 / 7),
                      rng.uniform(0.25 / 9, 0.5 - 0.25 / 9)])
        got = o.gather(G, U, p)
        want = [_trilinear_poly(p[0], p[1], p[2], coefs[q]) for q in range(3)]
        assert np.allclose(got, want, rtol=0, atol=1e-12)


def test_gather_matches_scipy_linear_interpolator_across_seam(oracle_mod):
    """Periodic trilinear interpolation equals scipy's RegularGridInterpolator on a padded copy."""
    from scipy.interpolate import RegularGridInterpolator

    o = oracle_mod
    n = 5
    G = o.make_grid(n)
    U = np.random.default_rng(1).standard_normal((n, n, n, 3))
    # pad one cell on each side periodically; axes ordered (x, y, z) for scipy
    Ux = np.transpose(U, (2, 1, 0, 3))
    P = np.pad(Ux, ((1, 1), (1, 1), (1, 1), (0, 0)), mode="wrap")
    ax = (np.arange(-1, n + 1) + 0.5) / n
    interp = RegularGridInterpolator((ax, ax, ax), P, method="linear")
    rng = np.random.default_rng(2)
    pts = rng.uniform(0.0, 1.0, (300, 3))
    pts[:50, 0] = rng.uniform(0.0, 0.5 / n, 50)       # near the lower seam
    pts[50:100, 1] = rng.uniform(1.0 - 0.5 / n, 1.0, 50)  # near the upper seam
    want = interp(pts)
    for p, w in zip(pts, want):
        assert np.allclose(o.gather(G, U, p), w, rtol=0, atol=1e-13)


def test_gather_at_cell_centres_returns_cell_value(oracle_mod):
    o = oracle_mod
    n = 4
    G = o.make_grid(n)
    U = np.random.default_rng(3).standard_normal((n, n, n, 3))
    for k in range(n):
        for j in range(n):
            for i in range(n):
                got = o.gather(G, U, [(i + 0.5) / n, (j + 0.5) / n, (k + 0.5) / n])
                assert np.allclose(got, U[k, j, i], rtol=0, atol=1e-15)


# --- wrap and cell index -----------------------------------------------------------------

def test_wrap_and_cell_match_exact_rational_arithmetic(oracle_mod):
    o = oracle_mod
    G = o.make_grid((8, 6, 10), L=(1.0, 0.75, 2.5))
    rng = np.random.default_rng(4)
    for _ in range(2000):
        x = [rng.uniform(-3, 4) * G.L[q] for q in range(3)]
        w = [o.wrap(x[q], G.L[q]) for q in range(3)]
        for q in range(3):
            assert 0.0 <= w[q] < G.L[q]
            # the wrapped value is x minus an integer number of periods, to rounding
            k = (Fraction(x[q]) - Fraction(w[q])) / Fraction(G.L[q])
            assert abs(k - round(k)) < 1e-12
        idx = o.cell(G, w)
        for q in range(3):
            h = Fraction(G.L[q]) / G.n[q]
            exact = min(int(math.floor(Fraction(w[q]) / h)), G.n[q] - 1)
            dist = min(abs(Fraction(w[q]) - h * exact), abs(Fraction(w[q]) - h * (exact + 1))) / h
            if dist > 1e-9:  # the comparison band of the cell rule
                assert idx[q] == exact
    # guards: images that round onto the upper boundary come back as 0
    assert o.wrap(-1e-300, 1.0) == 0.0
    assert o.wrap(1.0, 1.0) == 0.0
    assert o.wrap(2.0, 1.0) == 0.0
    assert o.cell(G, [0.0, 0.0, 0.0]) == (0, 0, 0)


# --- deposit and momentum balance (Sec. 2.1, Eq. 11; Sec. 2.5) -----------------------------

def test_momentum_balance_is_exact(oracle_mod):
    """sum_p m (v_T - v_0) - (sum_p m) g T + sum_c J_c = 0 (drag is internal to the mixture)."""
    o = oracle_mod
    n = 16
    G = o.make_grid(n)
    U = inputs.taylor_green(n)
    pos, vel, d, _ = inputs.particles(7, 0, 2000, vmax=0.5)
    T_steps, dt = 60, 1e-3
    p1, v1, src, _ = o.run(G, U, pos, vel, d, T_steps, dt)
    m = np.array([o.mass(G, x) for x in d])
    g = np.array([0.0, 0.0, -9.81])
    balance = (m[None, :] * (v1 - vel)).sum(1) - m.sum() * g * T_steps * dt + src.sum(1)
    scale = (m[None, :] * (np.abs(v1 - vel) + np.abs(g)[:, None] * T_steps * dt)).sum(1)
    assert np.all(np.abs(balance) <= 1e-12 * scale)
    inv = o.invariants(G, v1, d, src)
    assert inv[0] == 2000
    assert np.allclose(inv[1:4], (m[None, :] * v1).sum(1), rtol=1e-13, atol=0)
    assert np.allclose(inv[4:7], src.sum(1), rtol=1e-13, atol=1e-30)
    assert math.isclose(inv[7], m.sum(), rel_tol=1e-13)


def test_deposit_bruteforce_in_uniform_flow(oracle_mod):
    """Per-cell sums rebuilt from the closed-form trajectory: start-of-step cell, fluid-gain sign."""
    o = oracle_mod
    n = 6
    u = np.array([0.9, -0.7, 0.4])
    G = o.make_grid(n)
    U = inputs.uniform_field(n, u)
    pos, vel, d, _ = inputs.particles(11, 0, 60, vmax=2.0)
    nsteps, dt = 12, 4e-3
    _, _, src, _ = o.run(G, U, pos, vel, d, nsteps, dt)
    g = np.array([0.0, 0.0, -9.81])
    want = np.zeros((3, n ** 3))
    h = 1.0 / n
    for p in range(d.shape[0]):
        a = 18 * 1.8e-5 / (1000.0 * d[p] ** 2)
        m = 1000.0 * math.pi * d[p] ** 3 / 6.0
        vinf = u + g / a

        def state(t):
            v = vinf + (vel[:, p] - vinf) * math.exp(-a * t)
            x = pos[:, p] + vinf * t + (vel[:, p] - vinf) * (-math.expm1(-a * t)) / a
            return x % 1.0, v

        for s in range(nsteps):
            x0, v0 = state(s * dt)
            _, v1 = state((s + 1) * dt)
            frac = x0 / h - np.floor(x0 / h)
            assert np.all(np.minimum(frac, 1 - frac) > 1e-7), "choose a seed away from faces"
            i, j, k = (np.floor(x0 / h).astype(int) % n)
            c = i + n * (j + n * k)
            want[:, c] += -m * ((v1 - v0) - g * dt)
    scale = np.abs(want).max()
    assert np.max(np.abs(src - want)) <= 1e-10 * scale


# --- ordering key and stable sort (Sec. 2.2) ----------------------------------------------

def test_key_hand_values(oracle_mod):
    pin = GOLDEN["chunk_keys_B8_n32"]
    G = oracle_mod.make_grid(pin["n"], chunk_edge=pin["chunk_edge"])
    for (i, j, k), want in pin["cells_and_keys"]:
        assert oracle_mod.key(G, i, j, k) == want


@pytest.mark.parametrize("n,B", [((16, 8, 24), 8), ((12, 12, 12), 4), ((32, 32, 32), 32), ((8, 8, 8), 1)])
def test_key_is_a_chunk_major_bijection(oracle_mod, n, B):
    o = oracle_mod
    G = o.make_grid(n, chunk_edge=B)
    keys = {}
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                keys[(i, j, k)] = o.key(G, i, j, k)
    vals = np.array(sorted(keys.values()))
    assert len(set(vals)) == len(vals)
    nch = [math.ceil(n[q] / B) for q in range(3)]
    assert vals.max() < nch[0] * nch[1] * nch[2] * B ** 3
    for (i, j, k), v in keys.items():
        chunk = i // B + nch[0] * (j // B + nch[1] * (k // B))
        assert v // B ** 3 == chunk  # chunk-major
    if B >= 2:  # every aligned 2x2x2 block inside a chunk is a run of 8 consecutive keys
        for k in range(0, n[2], 2):
            for j in range(0, n[1], 2):
                for i in range(0, n[0], 2):
                    blk = sorted(keys[(i + a, j + b, k + c)] for a in (0, 1) for b in (0, 1) for c in (0, 1))
                    assert blk == list(range(blk[0], blk[0] + 8)) and blk[0] % 8 == 0


def test_stable_sort_matches_numpy_stable_argsort(oracle_mod):
    rng = np.random.default_rng(5)
    for n in (0, 1, 7, 1000, 20011):
        keys = rng.integers(0, 50, n).astype(np.uint32)
        perm = oracle_mod.sort_perm(keys)
        assert np.array_equal(perm, np.argsort(keys, kind="stable"))


def test_cell_counts_match_bincount(oracle_mod):
    o = oracle_mod
    G = o.make_grid((8, 4, 6))
    pos, _, _, _ = inputs.particles(3, 0, 5000)
    cnt = o.cell_counts(G, pos)
    idx = np.floor(pos * np.array([8, 4, 6])[:, None]).astype(int)
    want = np.bincount(idx[0] + 8 * (idx[1] + 4 * idx[2]), minlength=8 * 4 * 6)
    assert np.array_equal(cnt, want) and cnt.sum() == 5000


# --- adjoint: central finite differences with the deposit cells held fixed -------------------

def _adjoint_case(o, n=6, npart=12, nsteps=8, dt=2e-3):
    G = o.make_grid(n, alpha=0.9)
    U = inputs.taylor_green(n) + 0.2 * np.random.default_rng(6).standard_normal((n, n, n, 3))
    pos, vel, d, _ = inputs.particles(21, 0, npart, vmax=0.3)
    d = d * 2.0  # include some slow-relaxing particles
    return G, U, pos, vel, d, nsteps, dt


def _loss(o, G, U, pos, vel, d, nsteps, dt, target, frozen):
    _, _, src, _ = o.run(G, U, pos, vel, d, nsteps, dt, frozen=frozen)
    r = src - target
    return 0.5 * float((r * r).sum()), src


def test_adjoint_matches_central_finite_differences(oracle_mod):
    o = oracle_mod
    G, U, pos, vel, d, nsteps, dt = _adjoint_case(o)
    _, _, src0, trace = o.run(G, U, pos, vel, d, nsteps, dt, trace=True)
    target = 0.7 * src0 + 1e-13 * np.random.default_rng(7).standard_normal(src0.shape)
    lam = src0 - target
    gd, ga, gU = o.adjoint(G, U, pos, vel, d, nsteps, dt, lam)
    eps = 1e-4
    # diameters (relative step)
    for p in range(d.shape[0]):
        dp, dm = d.copy(), d.copy()
        dp[p] *= 1 + eps
        dm[p] *= 1 - eps
        fd = (_loss(o, G, U, pos, vel, dp, nsteps, dt, target, trace)[0]
              - _loss(o, G, U, pos, vel, dm, nsteps, dt, target, trace)[0]) / (2 * eps * d[p])
        assert abs(fd - gd[p]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gd).max())
    # drag scale (absolute step)
    Gp, Gm = o.make_grid(G.n[0], alpha=0.9 + eps), o.make_grid(G.n[0], alpha=0.9 - eps)
    fd = (_loss(o, Gp, U, pos, vel, d, nsteps, dt, target, trace)[0]
          - _loss(o, Gm, U, pos, vel, d, nsteps, dt, target, trace)[0]) / (2 * eps)
    assert abs(fd - ga) <= 1e-5 * abs(fd)
    # fluid field components with the largest gradients (absolute step)
    flat = np.argsort(-np.abs(gU).ravel())[:12]
    for f in flat:
        Up, Um = U.copy().reshape(-1), U.copy().reshape(-1)
        Up[f] += eps
        Um[f] -= eps
        fd = (_loss(o, G, Up.reshape(U.shape), pos, vel, d, nsteps, dt, target, trace)[0]
              - _loss(o, G, Um.reshape(U.shape), pos, vel, d, nsteps, dt, target, trace)[0]) / (2 * eps)
        assert abs(fd - gU.ravel()[f]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gU).max())


def test_adjoint_dot_product_with_random_direction(oracle_mod):
    """<grad, delta> equals the directional derivative of a linear functional of Jtot."""
    o = oracle_mod
    G, U, pos, vel, d, nsteps, dt = _adjoint_case(o, n=5, npart=20, nsteps=6)
    _, _, _, trace = o.run(G, U, pos, vel, d, nsteps, dt, trace=True)
    rng = np.random.default_rng(8)
    lam = rng.standard_normal((3, 5 ** 3))
    gd, ga, gU = o.adjoint(G, U, pos, vel, d, nsteps, dt, lam)
    dd = rng.standard_normal(d.shape) * d
    dU = rng.standard_normal(U.shape)
    da = 0.3
    eps = 1e-5

    def F(t):
        Gt = o.make_grid(5, alpha=0.9 + t * da)
        _, _, src, _ = o.run(Gt, U + t * dU, pos, vel, d + t * dd, nsteps, dt, frozen=trace)
        return float((lam * src).sum())

    fd = (F(eps) - F(-eps)) / (2 * eps)
    ip = float((gd * dd).sum() + ga * da + (gU.reshape(U.shape) * dU).sum())
    assert abs(fd - ip) <= 1e-6 * abs(fd)


# --- adjoint through the cloud-in-cell deposit: central differences with nothing held fixed ----

def test_adjoint_cic_matches_central_finite_differences_unfrozen(oracle_mod):
    """With the cloud-in-cell deposit the loss is continuous in the positions, so the adjoint, which
    then differentiates the deposit weights as well, matches central differences of the full run
    with no deposit cell held fixed."""
    o = oracle_mod
    G0, U, pos, vel, d, nsteps, dt = _adjoint_case(o)
    G = o.make_grid(G0.n[0], alpha=0.9, deposit="cic")
    _, _, src0, _ = o.run(G, U, pos, vel, d, nsteps, dt)
    target = 0.7 * src0 + 1e-13 * np.random.default_rng(17).standard_normal(src0.shape)
    lam = src0 - target
    gd, ga, gU = o.adjoint(G, U, pos, vel, d, nsteps, dt, lam)
    eps = 1e-4
    for p in range(d.shape[0]):
        dp, dm = d.copy(), d.copy()
        dp[p] *= 1 + eps
        dm[p] *= 1 - eps
        fd = (_loss(o, G, U, pos, vel, dp, nsteps, dt, target, None)[0]
              - _loss(o, G, U, pos, vel, dm, nsteps, dt, target, None)[0]) / (2 * eps * d[p])
        assert abs(fd - gd[p]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gd).max())
    Gp = o.make_grid(G.n[0], alpha=0.9 + eps, deposit="cic")
    Gm = o.make_grid(G.n[0], alpha=0.9 - eps, deposit="cic")
    fd = (_loss(o, Gp, U, pos, vel, d, nsteps, dt, target, None)[0]
          - _loss(o, Gm, U, pos, vel, d, nsteps, dt, target, None)[0]) / (2 * eps)
    assert abs(fd - ga) <= 1e-5 * abs(fd)
    flat = np.argsort(-np.abs(gU).ravel())[:12]
    for f in flat:
        Up, Um = U.copy().reshape(-1), U.copy().reshape(-1)
        Up[f] += eps
        Um[f] -= eps
        fd = (_loss(o, G, Up.reshape(U.shape), pos, vel, d, nsteps, dt, target, None)[0]
              - _loss(o, G, Um.reshape(U.shape), pos, vel, d, nsteps, dt, target, None)[0]) / (2 * eps)
        assert abs(fd - gU.ravel()[f]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gU).max())


def test_adjoint_cic_dot_product_with_random_direction(oracle_mod):
    """<grad, delta> equals the directional derivative of a linear functional of Jtot under the
    cloud-in-cell deposit, with nothing held fixed."""
    o = oracle_mod
    _, U, pos, vel, d, nsteps, dt = _adjoint_case(o, n=5, npart=20, nsteps=6)
    G = o.make_grid(5, alpha=0.9, deposit="cic")
    rng = np.random.default_rng(18)
    lam = rng.standard_normal((3, 5 ** 3))
    gd, ga, gU = o.adjoint(G, U, pos, vel, d, nsteps, dt, lam)
    dd = rng.standard_normal(d.shape) * d
    dU = rng.standard_normal(U.shape)
    da = 0.3
    eps = 1e-5

    def F(t):
        Gt = o.make_grid(5, alpha=0.9 + t * da, deposit="cic")
        _, _, src, _ = o.run(Gt, U + t * dU, pos, vel, d + t * dd, nsteps, dt)
        return float((lam * src).sum())

    fd = (F(eps) - F(-eps)) / (2 * eps)
    ip = float((gd * dd).sum() + ga * da + (gU.reshape(U.shape) * dU).sum())
    assert abs(fd - ip) <= 1e-6 * abs(fd)


def test_adjoint_cic_differs_from_the_cell_deposit_adjoint(oracle_mod):
    """The two deposits give different gradients for the same loss (the cloud-in-cell one is not
    the cell one under another name), and other physics are refused."""
    o = oracle_mod
    G0, U, pos, vel, d, nsteps, dt = _adjoint_case(o)
    G = o.make_grid(G0.n[0], alpha=0.9, deposit="cic")
    lam = np.random.default_rng(19).standard_normal((3, G0.n[0] ** 3))
    g_cic = o.adjoint(G, U, pos, vel, d, nsteps, dt, lam)[0]
    g_cell = o.adjoint(G0, U, pos, vel, d, nsteps, dt, lam)[0]
    assert np.abs(g_cic - g_cell).max() > 1e-3 * np.abs(g_cell).max()
    with pytest.raises(ValueError):
        o.adjoint(o.make_grid(G0.n[0], deposit="cic", drag="schiller_naumann"), U, pos, vel, d, nsteps, dt, lam)


def test_chunk_bounds_hand_example_and_properties(oracle_mod):
    """Chunk boxes (Sec. 2.2): a hand-worked example on a 16^3 grid with 8^3-cell chunks (box 1, h =
    1/16, chunk centres at 0.25 / 0.75), including a particle that crossed the periodic face and is
    unwrapped to the image nearest its chunk's centre; and, for particles that have not moved, every
    box lies inside its chunk's block of cells and does not depend on the particles' order."""
    G = oracle_mod.make_grid(16, chunk_edge=8)
    sort_pos = np.array([[0.01, 0.30, 0.90], [0.01, 0.20, 0.90], [0.01, 0.10, 0.95]])
    now_pos = np.array([[0.99, 0.35, 0.02], [0.01, 0.20, 0.90], [0.01, 0.10, 0.95]])
    b = oracle_mod.chunk_bounds(G, sort_pos, now_pos)
    # chunk 0 holds particles 0 and 1: particle 0 moved from x = 0.01 across the face to 0.99,
    # which is x = -0.01 next to the chunk (centre 0.25)
    assert np.allclose(b[0], [-0.01, 0.01, 0.01, 0.35, 0.20, 0.10], atol=1e-15)
    # chunk (1, 1, 1) = 1 + 2 (1 + 2 * 1) = 7 holds particle 2, at x = 0.02 -> 1.02 beside centre 0.75
    assert np.allclose(b[7], [1.02, 0.90, 0.95, 1.02, 0.90, 0.95], atol=1e-15)
    assert np.all(np.isinf(b[[1, 2, 3, 4, 5, 6]]))
    rng = np.random.default_rng(9)
    pos = rng.uniform(0, 1, size=(3, 500))
    bb = oracle_mod.chunk_bounds(G, pos, pos)
    perm = rng.permutation(500)
    assert np.array_equal(bb, oracle_mod.chunk_bounds(G, pos[:, perm], pos[:, perm]))
    for c in range(8):
        lo = np.array([c % 2, (c // 2) % 2, c // 4]) * 0.5
        assert np.all(bb[c, :3] >= lo) and np.all(bb[c, 3:] <= lo + 0.5)


def test_blocked_all_cores_run_is_deterministic(oracle_mod):
    """The all-cores oracle (fixed particle blocks, partial sources added in block order): independent of
    the thread count bit for bit, identical to the single-thread run when one block holds every particle,
    the same particle states for any block size, and sources equal to the single-thread run's up to the
    rounding of the changed summation order."""
    from paper_2603_26691_gb300 import inputs

    o = oracle_mod
    G = o.make_grid(12)
    U = inputs.random_fourier(12, seed=4)
    n, steps, dt = 9_001, 6, 5e-4
    pos, vel, d, _ = inputs.particles(21, 0, n, vmax=0.2)
    part = lambda f, c: (pos[:, f:f + c], vel[:, f:f + c], d[f:f + c])  # noqa: E731
    p0, v0, s0, _ = o.run(G, U, pos, vel, d, steps, dt)
    states = {}

    def keep(first, p, v):
        states[first] = (p, v)

    s1 = o.run_blocked(G, U, part, n, steps, dt, block=1000, threads=1, keep=keep)
    s4 = o.run_blocked(G, U, part, n, steps, dt, block=1000, threads=4)
    assert np.array_equal(s1, s4)
    p1 = np.concatenate([states[f][0] for f in sorted(states)], axis=1)
    v1 = np.concatenate([states[f][1] for f in sorted(states)], axis=1)
    assert np.array_equal(p1, p0) and np.array_equal(v1, v0)
    assert np.abs(s1 - s0).max() <= 1e-13 * np.abs(s0).max()
    sall = o.run_blocked(G, U, part, n, steps, dt, block=n, threads=3)
    assert np.array_equal(sall, s0)


def test_blocked_adjoint_matches_the_single_run(oracle_mod):
    """The all-cores adjoint (fixed blocks, gradients added in block order) equals the single-thread
    adjoint up to the rounding of the changed summation order, and is independent of the thread count."""
    from paper_2603_26691_gb300 import inputs

    o = oracle_mod
    G = o.make_grid(8)
    U = inputs.random_fourier(8, seed=6)
    n, steps, dt = 1_201, 5, 1e-3
    pos, vel, d, _ = inputs.particles(31, 0, n, vmax=0.1)
    lam = np.random.default_rng(4).standard_normal((3, 512))
    gd0, ga0, gU0 = o.adjoint(G, U, pos, vel, d, steps, dt, lam)
    part = lambda f, c: (pos[:, f:f + c], vel[:, f:f + c], d[f:f + c])  # noqa: E731
    gds = {}
    ga1, gU1 = o.adjoint_blocked(G, U, part, n, steps, dt, lam, block=300, threads=1,
                                 keep=lambda f, g: gds.__setitem__(f, g))
    ga4, gU4 = o.adjoint_blocked(G, U, part, n, steps, dt, lam, block=300, threads=4)
    assert ga1 == ga4 and np.array_equal(gU1, gU4)
    assert np.array_equal(np.concatenate([gds[f] for f in sorted(gds)]), gd0)
    assert abs(ga1 - ga0) <= 1e-13 * abs(ga0)
    assert np.abs(gU1 - gU0).max() <= 1e-13 * np.abs(gU0).max()
