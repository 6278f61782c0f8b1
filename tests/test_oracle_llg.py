"""Pins of the FP64 field / LLG / energy oracle (oracle/llg.py) against
closed forms: Neumann-Laplacian eigenmodes, the energy-field identity
H = -(1/(mu0 V)) dE/dM, the exact macrospin solution of Eq. (6), |M| = Ms,
and monotone energy decay for alpha > 0."""
import numpy as np
import pytest

from oracle import tensor as T
from oracle import demag as D
from oracle import llg as L
from paper_1406_7459_gb300 import inputs

MU0 = T.MU0


def test_uniform_state_has_no_exchange_field():
    M = inputs.uniform_m((5, 4, 3), 8.6e5, (0.3, 0.4, 0.5)).astype(np.float64)
    H = L.h_exchange(M, (5e-9, 4e-9, 3e-9), 8.6e5, 1.3e-11)
    assert np.max(np.abs(H)) < 1e-6


@pytest.mark.parametrize("q", [(1, 0, 0), (2, 1, 0), (3, 2, 1)])
def test_neumann_cosine_modes_are_exact_eigenvectors(q):
    grid, cell = (8, 6, 4), (5e-9, 4e-9, 3e-9)
    Ms, A = 8.6e5, 1.3e-11
    nx, ny, nz = grid
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                          indexing="ij")
    mode = (np.cos(np.pi * q[0] * (i + 0.5) / nx)
            * np.cos(np.pi * q[1] * (j + 0.5) / ny)
            * np.cos(np.pi * q[2] * (k + 0.5) / nz))
    M = np.stack([mode, 0.5 * mode, -mode])
    lam = sum((2 - 2 * np.cos(np.pi * qa / na)) / d ** 2
              for qa, na, d in zip(q, grid, cell))
    H = L.h_exchange(M, cell, Ms, A)
    expect = -(2 * A / (MU0 * Ms * Ms)) * lam * M
    assert np.max(np.abs(H - expect)) < 1e-10 * np.max(np.abs(expect))


def _energy(M, cell, Ms, A, Ku, Hext, Kt, Lp):
    Hd = D.demag_fft(M, Kt, Lp)
    return L.energy_terms(M, Hd, cell, Ms, A, Ku, Hext)[0]


def test_effective_field_is_minus_energy_gradient():
    """dE = -mu0 V sum H_eff . dM for every term of Eq. (1)/(2), checked by
    central differences in a random direction (M off the sphere is fine)."""
    grid, cell = (6, 5, 3), (5e-9, 4e-9, 3e-9)
    Ms, A, Ku, Hext = 8.6e5, 1.3e-11, 4e4, (1e4, -2e4, 3e4)
    V = np.prod(cell)
    M = inputs.random_unit_m(grid, Ms, seed=11).astype(np.float64)
    dM = inputs.random_unit_m(grid, Ms, seed=12).astype(np.float64)
    Lp = D.default_lengths(grid)
    Kt = D.kernel_spectrum(T.tensor_octant(grid, cell), Lp)
    eps = 1e-4
    dE = (_energy(M + eps * dM, cell, Ms, A, Ku, Hext, Kt, Lp)
          - _energy(M - eps * dM, cell, Ms, A, Ku, Hext, Kt, Lp)) / (2 * eps)
    H = L.h_effective(M, cell, Ms, A, Ku, Hext, D.demag_fft(M, Kt, Lp))
    expect = -MU0 * V * np.sum(H * dM)
    assert abs(dE - expect) < 1e-8 * abs(expect)


def test_exchange_link_energy_identity():
    grid, cell = (7, 5, 2), (5e-9, 4e-9, 3e-9)
    Ms, A = 8.6e5, 1.3e-11
    M = inputs.random_unit_m(grid, Ms, seed=5).astype(np.float64)
    E = L.energy_terms(M, np.zeros_like(M), cell, Ms, A, 0.0, (0, 0, 0))
    Hx = L.h_exchange(M, cell, Ms, A)
    assert abs(E[1] + 0.5 * MU0 * np.prod(cell) * np.sum(Hx * M)) < 1e-12 * abs(E[1])


def test_llg_rhs_is_perpendicular_to_m():
    grid = (4, 3, 2)
    M = inputs.random_unit_m(grid, 8.6e5, seed=1).astype(np.float64)
    H = 1e5 * inputs.random_unit_m(grid, 1.0, seed=2).astype(np.float64)
    f = L.llg_rhs(M, H, 8.6e5, 0.3, 2.211e5)
    assert np.max(np.abs(np.sum(f * M, axis=0))) < 1e-9 * np.max(np.abs(f)) * 8.6e5


def _macrospin_run(dt, t_end, theta0, phi0, Hz, alpha, gamma, Ms):
    cell = (3e-9, 3e-9, 3e-9)          # cube: demag field is parallel to M
    grid = (1, 1, 1)
    Lp = D.default_lengths(grid)
    Kt = D.kernel_spectrum(T.tensor_octant(grid, cell), Lp)
    M = Ms * np.array([np.sin(theta0) * np.cos(phi0),
                       np.sin(theta0) * np.sin(phi0),
                       np.cos(theta0)]).reshape(3, 1, 1, 1)
    n = int(round(t_end / dt))
    M = L.run_euler(M, n, dt, cell, Ms, 1.3e-11, 0.0, alpha, gamma,
                    (0.0, 0.0, Hz), Kt, Lp)
    return M.reshape(3) / Ms


def test_macrospin_matches_closed_form_with_first_order_error():
    theta0, phi0, Hz, alpha, gamma, Ms = 1.2, 0.3, 2e5, 0.1, 2.211e5, 8.6e5
    t_end = 2e-10
    th, ph = L.macrospin_closed_form(theta0, phi0, Hz, alpha, gamma, t_end)
    exact = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    errs = []
    for dt in (4e-14, 2e-14, 1e-14):
        m = _macrospin_run(dt, t_end, theta0, phi0, Hz, alpha, gamma, Ms)
        errs.append(np.linalg.norm(m - exact))
    assert errs[-1] < 5e-3
    for a, b in zip(errs[:-1], errs[1:]):
        assert 1.8 < a / b < 2.2, errs        # forward Euler: O(dt)


def test_renormalisation_keeps_norm_and_energy_decays():
    grid, cell = (8, 8, 2), (5e-9, 5e-9, 3e-9)
    Ms, A, Ku, alpha, gamma = 8.6e5, 1.3e-11, 5e2, 0.5, 2.211e5
    Hext = (1e4, 2e3, 0.0)
    Lp = D.default_lengths(grid)
    Kt = D.kernel_spectrum(T.tensor_octant(grid, cell), Lp)
    M = inputs.random_unit_m(grid, Ms, seed=1).astype(np.float64)
    E_prev = _energy(M, cell, Ms, A, Ku, Hext, Kt, Lp)
    for _ in range(60):
        M, _ = L.euler_step(M, 1e-13, cell, Ms, A, Ku, alpha, gamma, Hext, Kt, Lp)
        assert np.max(np.abs(np.sqrt(np.sum(M * M, axis=0)) - Ms)) < 1e-9 * Ms
        E = _energy(M, cell, Ms, A, Ku, Hext, Kt, Lp)
        assert E <= E_prev + 1e-12 * abs(E_prev)
        E_prev = E


def test_undamped_energy_drift_is_first_order():
    grid, cell = (6, 6, 1), (5e-9, 5e-9, 3e-9)
    Ms, A, Ku, gamma = 8.6e5, 1.3e-11, 0.0, 2.211e5
    Lp = D.default_lengths(grid)
    Kt = D.kernel_spectrum(T.tensor_octant(grid, cell), Lp)
    M0 = inputs.perturbed_m(grid, Ms, seed=4, amplitude=0.3).astype(np.float64)
    E0 = _energy(M0, cell, Ms, A, Ku, (0, 0, 0), Kt, Lp)
    drift = []
    for dt, n in ((2e-15, 100), (1e-15, 200)):
        M = L.run_euler(M0, n, dt, cell, Ms, A, Ku, 0.0, gamma, (0, 0, 0), Kt, Lp)
        drift.append(abs(_energy(M, cell, Ms, A, Ku, (0, 0, 0), Kt, Lp) - E0))
    assert 1.6 < drift[0] / drift[1] < 2.4, drift


def _macrospin_rk(method, dt, t_end, theta0, phi0, Hz, alpha, gamma, Ms):
    cell = (3e-9, 3e-9, 3e-9)
    grid = (1, 1, 1)
    Lp = D.default_lengths(grid)
    Kt = D.kernel_spectrum(T.tensor_octant(grid, cell), Lp)
    M = Ms * np.array([np.sin(theta0) * np.cos(phi0), np.sin(theta0) * np.sin(phi0),
                       np.cos(theta0)]).reshape(3, 1, 1, 1)
    n = int(round(t_end / dt))
    M = L.run_rk(M, n, dt, method, cell, Ms, 1.3e-11, 0.0, alpha, gamma, (0.0, 0.0, Hz), Kt, Lp)
    return M.reshape(3) / Ms


@pytest.mark.parametrize("method,order", [("euler", 1), ("heun", 2), ("rk4", 4)])
def test_runge_kutta_orders_on_the_macrospin(method, order):
    """Error against the closed-form solution of Eq. (6) falls as dt^order."""
    theta0, phi0, Hz, alpha, gamma, Ms = 1.2, 0.3, 2e5, 0.1, 2.211e5, 8.6e5
    t_end = 2e-10
    th, ph = L.macrospin_closed_form(theta0, phi0, Hz, alpha, gamma, t_end)
    exact = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    dts = (8e-13, 4e-13, 2e-13) if order == 4 else (4e-14, 2e-14, 1e-14)
    errs = [np.linalg.norm(_macrospin_rk(method, dt, t_end, theta0, phi0, Hz, alpha, gamma, Ms) - exact)
            for dt in dts]
    ratios = [a / b for a, b in zip(errs[:-1], errs[1:])]
    for r in ratios:
        assert 0.8 * 2 ** order < r < 1.25 * 2 ** order, (errs, ratios)


def test_rk_euler_branch_equals_euler_step():
    grid, cell = (5, 4, 2), (5e-9, 5e-9, 3e-9)
    Ms, A, Ku, alpha, gamma, Hext = 8.6e5, 1.3e-11, 1e4, 0.3, 2.211e5, (1e4, 0, 0)
    Lp = D.default_lengths(grid)
    Kt = D.kernel_spectrum(T.tensor_octant(grid, cell), Lp)
    M = inputs.random_unit_m(grid, Ms, seed=3).astype(np.float64)
    a = L.rk_step(M, 1e-13, "euler", cell, Ms, A, Ku, alpha, gamma, Hext, Kt, Lp)
    b, _ = L.euler_step(M, 1e-13, cell, Ms, A, Ku, alpha, gamma, Hext, Kt, Lp)
    assert np.max(np.abs(a - b)) < 1e-9 * Ms


# ---- adaptive Dormand-Prince integrator (beyond the paper's Euler scheme)

def test_dormand_prince_tableau_order_conditions():
    """Row sums equal the nodes; the fifth-order weights satisfy the order
    conditions up to order 5 (the ones for bushy and tall trees checked here),
    the embedded weights b - e those up to order 4 but not the order-5
    quadrature condition."""
    from fractions import Fraction
    c, A, b, e = L.DP_C, L.DP_A, L.DP_B, L.DP_E
    for i in range(1, 6):
        assert abs(sum(A[i]) - c[i]) < 1e-15
    a = lambda i, j: A[i][j] if i < 6 and j < len(A[i]) else (b[j] if i == 6 else 0.0)
    bh = [bi - ei for bi, ei in zip(b, e)]
    for w, top in ((b, 5), (bh, 4)):
        for q in range(1, top + 1):
            assert abs(sum(wi * ci ** (q - 1) for wi, ci in zip(w, c)) - 1.0 / q) < 1e-14, (top, q)
        # sum_i w_i sum_j a_ij c_j = 1/6, sum_i w_i c_i sum_j a_ij c_j = 1/8
        s6 = sum(w[i] * sum(a(i, j) * c[j] for j in range(i)) for i in range(7))
        s8 = sum(w[i] * c[i] * sum(a(i, j) * c[j] for j in range(i)) for i in range(7))
        s12 = sum(w[i] * sum(a(i, j) * c[j] ** 2 for j in range(i)) for i in range(7))
        assert abs(s6 - 1.0 / 6.0) < 1e-14 and abs(s8 - 1.0 / 8.0) < 1e-14 and abs(s12 - 1.0 / 12.0) < 1e-14
    # the embedded pair is genuinely of order 4: its order-5 quadrature fails
    assert abs(sum(wi * ci ** 4 for wi, ci in zip(bh, c)) - 0.2) > 1e-4
    assert Fraction(e[6]).limit_denominator(100) == Fraction(-1, 40)


def _macrospin_setup(theta0, phi0, Ms):
    cell = (3e-9, 3e-9, 3e-9)
    Lp = D.default_lengths((1, 1, 1))
    Kt = D.kernel_spectrum(T.tensor_octant((1, 1, 1), cell), Lp)
    M = Ms * np.array([np.sin(theta0) * np.cos(phi0), np.sin(theta0) * np.sin(phi0),
                       np.cos(theta0)]).reshape(3, 1, 1, 1)
    return cell, Kt, Lp, M


def test_dormand_prince_fixed_step_order_and_error_estimate():
    """Fixed steps on the macrospin: the global error against the closed form
    falls as dt^5, and the step's error estimate (the fourth-order local
    error) as dt^5."""
    theta0, phi0, Hz, alpha, gamma, Ms = 1.2, 0.3, 2e5, 0.1, 2.211e5, 8.6e5
    cell, Kt, Lp, M0 = _macrospin_setup(theta0, phi0, Ms)
    args = (cell, Ms, 1.3e-11, 0.0, alpha, gamma, (0.0, 0.0, Hz), Kt, Lp)
    t_end = 2e-10
    th, ph = L.macrospin_closed_form(theta0, phi0, Hz, alpha, gamma, t_end)
    exact = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    errs, ests = [], []
    for dt in (4e-12, 2e-12, 1e-12):
        M = M0.copy()
        k1 = L._rhs(M, *args)
        first_est = None
        for _ in range(int(round(t_end / dt))):
            M, est, k1 = L.dopri5_step(M, k1, dt, *args)
            if first_est is None:
                first_est = est
        errs.append(np.linalg.norm(M.reshape(3) / Ms - exact))
        ests.append(first_est)
    for r in (errs[0] / errs[1], errs[1] / errs[2]):
        assert 0.75 * 32 < r < 1.3 * 32, errs
    for r in (ests[0] / ests[1], ests[1] / ests[2]):
        assert 0.75 * 32 < r < 1.3 * 32, ests


def test_dormand_prince_adaptive_run_meets_tolerance():
    """Adaptive runs on the macrospin end within a small multiple of tol of
    the closed form, and a tighter tol takes more steps, about
    tol^(-1/5) more."""
    theta0, phi0, Hz, alpha, gamma, Ms = 1.2, 0.3, 2e5, 0.1, 2.211e5, 8.6e5
    cell, Kt, Lp, M0 = _macrospin_setup(theta0, phi0, Ms)
    t_end = 4e-10
    th, ph = L.macrospin_closed_form(theta0, phi0, Hz, alpha, gamma, t_end)
    exact = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    steps = []
    for tol in (1e-6, 1e-8):
        M, dt_next, (acc, rej, nev, t) = L.run_dopri5(M0.copy(), t_end, 1e-13, tol, 10000, cell, Ms, 1.3e-11, 0.0,
                                                      alpha, gamma, (0.0, 0.0, Hz), Kt, Lp)
        assert abs(t - t_end) < 1e-12 * t_end
        assert nev == 1 + 6 * (acc + rej)
        err = np.linalg.norm(M.reshape(3) / Ms - exact)
        assert err < 50 * tol * acc, (tol, err, acc)
        steps.append(acc)
    assert 100 ** 0.2 * 0.6 < steps[1] / steps[0] < 100 ** 0.2 * 1.6, steps


def test_dormand_prince_controller_factors():
    assert L.dp_next_factor(0.0, 1e-6, False) == L.DP_FMAX
    assert L.dp_next_factor(1e-1, 1e-6, False) == L.DP_FMIN
    assert L.dp_next_factor(1e-9, 1e-6, True) == 1.0
    assert abs(L.dp_next_factor(1e-6, 1e-6, False) - 0.9) < 1e-15
