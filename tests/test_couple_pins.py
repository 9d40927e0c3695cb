"""Pins of the oracle's asynchronous two-way coupling (Sec. 2.3) and extrapolator-corrector method
(Sec. 2.4, Eqs. 12-14), checked against what the mathematics fixes: exactness of the extrapolators
on steady and linear-in-time sources, conservation over time, the eigenmode solution of the
implicit diffusion step and of its Jacobi iteration, the two-body closed form of a particle
exchanging momentum with a uniform fluid (first-order convergence in the coupling interval), and
the global momentum budget."""
import numpy as np
import pytest

import oracle
from paper_2603_26691_gb300 import inputs


def _estimates(extrap, S):
    """S_est^n for n = 0..N-1 from the oracle, given the sources S[n] of every interval."""
    out = []
    for n in range(len(S)):
        prev = [S[n - k] if n - k >= 0 else None for k in (1, 2, 3)]
        out.append(oracle.ecm_estimate(extrap, *prev, m=S[0].size))
    return np.array(out)


def test_zero_extrapolator_is_a_lag_of_one_interval():
    rng = np.random.default_rng(0)
    S = rng.normal(size=(7, 11))
    est = _estimates("zero", S)
    assert np.array_equal(est[0], np.zeros(11))
    assert np.array_equal(est[1:], S[:-1])


@pytest.mark.parametrize("extrap", ["const", "lin"])
def test_extrapolators_are_exact_on_the_data_they_model(extrap):
    # a steady source is reproduced by the constant extrapolator from the second interval on, and
    # a source linear in time by the linear one from the third (the estimate then equals S^n)
    n = np.arange(9)[:, None]
    S = (0.7 + 0.0 * n) * np.ones((9, 5)) if extrap == "const" else (0.3 + 0.25 * n) * np.ones((9, 5))
    est = _estimates(extrap, S)
    first = 2 if extrap == "const" else 3
    assert np.abs(est[first:] - S[first:]).max() <= 1e-14


@pytest.mark.parametrize("extrap", ["zero", "const", "lin"])
def test_estimates_are_conservative_over_time(extrap):
    # what the fluid has received never drifts from what the particles gave: the running
    # difference only involves the last three intervals, whatever the history
    rng = np.random.default_rng(1)
    S = rng.normal(size=(40, 6))
    est = _estimates(extrap, S)
    lag = np.cumsum(S, axis=0) - np.cumsum(est, axis=0)
    # bounded by a few source magnitudes at every N (no accumulation)
    assert np.abs(lag).max() <= 8 * np.abs(S).max()
    # and the same as the oracle's pending sources after N intervals with no particles moving
    # anything: checked through orc_couple below in the momentum budget


def _mode(G, kvec, amp=1.0):
    """A single sine eigenmode of the periodic 7-point Laplacian in every component."""
    x, y, z = inputs.cell_centres(tuple(G.n), tuple(G.L))
    phase = 2 * np.pi * (kvec[0] * x / G.L[0] + kvec[1] * y / G.L[1] + kvec[2] * z / G.L[2])
    U = np.zeros(x.shape + (3,))
    for q in range(3):
        U[..., q] = amp * (q + 1) * np.sin(phase)
    return U


@pytest.mark.parametrize("sweeps", [1, 10, 300])
def test_jacobi_on_an_eigenmode_matches_its_closed_form(sweeps):
    # for an eigenmode of the discrete Laplacian with eigenvalue -sum_q (2/h_q^2)(1 - cos(2 pi k_q / n_q)),
    # the implicit step divides it by 1 + s (s = nu dtc times that), and Jacobi from u* converges
    # to that fixed point with the factor rho = (2 sum lam_q cos(2 pi k_q/n_q)) / (1 + 2 sum lam_q)
    G = oracle.make_grid((12, 10, 8), L=(1.0, 0.8, 1.3))
    nu, dtc = 2e-3, 0.05
    k = (2, 1, 3)
    U0 = _mode(G, k)
    h = np.array(G.L) / np.array(G.n)
    lam = nu * dtc / h ** 2
    cosk = np.cos(2 * np.pi * np.array(k) / np.array(G.n))
    s = np.sum(2 * lam * (1 - cosk))
    rho = np.sum(2 * lam * cosk) / (1 + 2 * lam.sum())
    fixed = U0 / (1 + s)
    expect = fixed + (U0 - fixed) * rho ** sweeps
    got = oracle.fluid_update(G, U0, None, 1.2, nu, dtc, sweeps)
    assert np.abs(got - expect).max() <= 1e-12 * np.abs(U0).max()


def test_fluid_update_conserves_momentum_and_adds_the_source():
    G = oracle.make_grid((8, 6, 10))
    rng = np.random.default_rng(2)
    U = rng.normal(size=(10, 6, 8, 3))
    S = rng.normal(size=(3, 480)) * 1e-7
    rho_f = 1.2
    V = np.prod(np.array(G.L) / np.array(G.n))
    got = oracle.fluid_update(G, U, S, rho_f, 1e-3, 5e-3, 10)
    want = U.reshape(-1, 3).sum(0) + S.sum(1) / (rho_f * V)
    assert np.abs(got.reshape(-1, 3).sum(0) - want).max() <= 1e-12 * np.abs(U).sum()


def _two_body(K, dt, extrap, nint):
    """One particle in a one-cell periodic box (the fluid velocity is uniform), no gravity."""
    G = oracle.make_grid(1, g=(0.0, 0.0, 0.0))
    d = np.array([50e-6])
    m = oracle.mass(G, d[0])
    tau = 1000.0 * d[0] ** 2 / (18 * 1.8e-5)
    rho_f = m / 1.0  # fluid mass M_f = rho_f * V = m (V = 1)
    U = np.zeros((1, 1, 1, 3))
    pos = np.array([[0.3], [0.4], [0.5]])
    vel = np.array([[1.0], [0.0], [0.0]])
    Uo, po, vo, pend = oracle.couple(G, U, pos, vel, d, nint, K, dt, rho_f, 0.0, 0, extrap)
    return G, m, tau, Uo, vo, pend


@pytest.mark.parametrize("extrap", ["zero", "const", "lin"])
def test_two_body_exchange_converges_at_first_order(extrap):
    # closed form (Sec. 4.1's test of a particle slowing down in quiescent fluid): with fluid mass
    # M_f, the relative velocity decays as exp(-(1 + m/M_f) t / tau) and m v + M_f u is constant
    errs = []
    T = 4e-3
    for K, dt in [(1, T / 16), (1, T / 32), (1, T / 64)]:
        G, m, tau, Uo, vo, pend = _two_body(K, dt, extrap, round(T / (K * dt)))
        w = np.exp(-(1 + 1.0) * T / tau)  # M_f = m
        u_exact = 0.5 * (1 - w)  # fluid velocity: (m v0 - m w v0) / (m + M_f)
        errs.append(abs(Uo.reshape(3)[0] - u_exact))
        # exact momentum budget at every resolution: particle + fluid + pending = m v0
        total = m * vo[0, 0] + m * Uo.reshape(3)[0] + pend[0, 0]
        assert abs(total - m * 1.0) <= 1e-12 * m
    ratios = [errs[i + 1] / errs[i] for i in range(len(errs) - 1)]
    assert all(0.35 <= r <= 0.65 for r in ratios), (errs, ratios)


@pytest.mark.parametrize("extrap", ["zero", "lin"])
def test_global_momentum_budget(extrap):
    # particles + fluid + sources not yet applied - gravity impulse is conserved exactly (FP64)
    N = 12
    G = oracle.make_grid(N)
    U = inputs.taylor_green(N) * 0.5
    pos, vel, d, _ = inputs.particles(17, 0, 400, vmax=0.2)
    rho_f = 1.2e-6  # a light fluid so that the exchange moves it noticeably
    K, dt, nint = 3, 1e-3, 7
    V = (1.0 / N) ** 3
    Uo, po, vo, pend = oracle.couple(G, U, pos, vel, d, nint, K, dt, rho_f, 1e-3, 10, extrap)
    m = np.array([oracle.mass(G, di) for di in d])
    g = np.array([0.0, 0.0, -9.81])
    P0 = (m * vel).sum(1) + rho_f * V * U.reshape(-1, 3).sum(0)
    P1 = (m * vo).sum(1) + rho_f * V * Uo.reshape(-1, 3).sum(0) + pend.sum(1)
    grav = m.sum() * g * nint * K * dt
    scale = np.abs(P0).max() + np.abs(grav).max() + np.abs(pend).sum()
    assert np.abs(P1 - P0 - grav).max() <= 1e-12 * scale
    # the fluid did move: the exchange is not negligible in this setup
    assert np.abs(Uo - U).max() > 1e-3
