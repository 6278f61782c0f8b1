"""Effective field, LLG right-hand side, Euler step, energy (FP64; test
infrastructure only).

Readings of the paper's Sec. 2:
* Eq. (1)'s exchange term repeats M_x three times; read as the sum over
  M_x, M_y, M_z.
* Eq. (3)/(4) omit mu0, which Eq. (5) carries; H_exch = 2A/(mu0 Ms^2) lap M
  is the dimensionally consistent field (A/m) from Eq. (1)-(2).
* Eq. (5) is read from Eq. (1): H_anis = -(2 Ku/(mu0 Ms^2)) (0, M_y, M_z),
  an easy x axis.
* Eq. (6) with ``gamma`` = gamma_0 in m/(A s) and H in A/m: the mu0 inside
  Eq. (6) is absorbed into gamma_0.
* Exchange boundary: free (Neumann): a missing neighbour is the cell itself.
* Integrator: forward Euler (Table 1 caption) with every term at M^n, then
  renormalisation |M| = Ms.
"""
import numpy as np

from .tensor import MU0
from .demag import demag_fft


def h_exchange(M, cell, Ms, A):
    """Eq. (4) for all three components, Neumann boundaries."""
    pref = 2.0 * A / (MU0 * Ms * Ms)
    P = np.pad(M, ((0, 0), (1, 1), (1, 1), (1, 1)), mode="edge")
    c = P[:, 1:-1, 1:-1, 1:-1]
    dx, dy, dz = cell
    lap = ((P[:, 1:-1, 1:-1, 2:] - 2 * c + P[:, 1:-1, 1:-1, :-2]) / dx ** 2
           + (P[:, 1:-1, 2:, 1:-1] - 2 * c + P[:, 1:-1, :-2, 1:-1]) / dy ** 2
           + (P[:, 2:, 1:-1, 1:-1] - 2 * c + P[:, :-2, 1:-1, 1:-1]) / dz ** 2)
    return pref * lap


def h_anisotropy(M, Ms, Ku):
    """Uniaxial anisotropy with easy axis x, from Eq. (1)-(2)."""
    pref = -2.0 * Ku / (MU0 * Ms * Ms)
    H = np.zeros_like(M, dtype=np.float64)
    H[1] = pref * M[1]
    H[2] = pref * M[2]
    return H


def h_effective(M, cell, Ms, A, Ku, H_ext, H_demag):
    """Eq. (2): H_eff = H_exch + H_anis + H_demag + H_ext."""
    H = h_exchange(M, cell, Ms, A) + h_anisotropy(M, Ms, Ku) + H_demag
    return H + np.asarray(H_ext, np.float64).reshape(3, 1, 1, 1)


def llg_rhs(M, H, Ms, alpha, gamma):
    """Eq. (6): dM/dt = -g/(1+a^2) M x H - a g/((1+a^2) Ms) M x (M x H)."""
    MxH = np.cross(M, H, axis=0)
    MxMxH = np.cross(M, MxH, axis=0)
    c = gamma / (1.0 + alpha * alpha)
    return -c * MxH - (c * alpha / Ms) * MxMxH


def euler_step(M, dt, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L):
    """One forward-Euler step of Eq. (6) with every field at M^n, followed by
    renormalisation to |M| = Ms.  Returns (M^{n+1}, H_demag(M^n))."""
    Hd = demag_fft(M, Kt, L)
    H = h_effective(M, cell, Ms, A, Ku, H_ext, Hd)
    Mn = M + dt * llg_rhs(M, H, Ms, alpha, gamma)
    Mn = Mn * (Ms / np.sqrt(np.sum(Mn * Mn, axis=0)))
    return Mn, Hd


def _rhs(M, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L):
    H = h_effective(M, cell, Ms, A, Ku, H_ext, demag_fft(M, Kt, L))
    return llg_rhs(M, H, Ms, alpha, gamma)


def rk_step(M, dt, method, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L):
    """One explicit Runge-Kutta step of Eq. (6), the paper's Euler scheme
    replaced by a higher-order one (beyond the paper).  Stage states are
    plain (not renormalised); the new state is renormalised to |M| = Ms as
    in the Euler step.
      heun: k1 = f(M), k2 = f(M + dt k1), M' = M + dt (k1 + k2)/2
      rk4:  k1 = f(M), k2 = f(M + dt/2 k1), k3 = f(M + dt/2 k2),
            k4 = f(M + dt k3), M' = M + dt (k1 + 2 k2 + 2 k3 + k4)/6"""
    f = lambda X: _rhs(X, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L)
    if method == "euler":
        Mn = M + dt * f(M)
    elif method == "heun":
        k1 = f(M)
        k2 = f(M + dt * k1)
        Mn = M + 0.5 * dt * (k1 + k2)
    elif method == "rk4":
        k1 = f(M)
        k2 = f(M + 0.5 * dt * k1)
        k3 = f(M + 0.5 * dt * k2)
        k4 = f(M + dt * k3)
        Mn = M + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    else:
        raise ValueError(method)
    return Mn * (Ms / np.sqrt(np.sum(Mn * Mn, axis=0)))


def run_rk(M, nsteps, dt, method, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L):
    for _ in range(nsteps):
        M = rk_step(M, dt, method, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L)
    return M


# Dormand-Prince embedded Runge-Kutta pair RK5(4) (Dormand and Prince,
# J. Comput. Appl. Math. 6 (1980) 19-26): nodes c, stage matrix a, fifth-
# order weights b, and e = b - b_hat, the difference to the embedded
# fourth-order weights (b_hat_7 = 1/40 acts on the stage at the new state).
DP_C = (0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0)
DP_A = (
    (),
    (1.0 / 5.0,),
    (3.0 / 40.0, 9.0 / 40.0),
    (44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0),
    (19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0),
    (9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0),
)
DP_B = (35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0.0)
DP_E = (71.0 / 57600.0, 0.0, -71.0 / 16695.0, 71.0 / 1920.0, -17253.0 / 339200.0, 22.0 / 525.0, -1.0 / 40.0)


def dopri5_step(M, k1, dt, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L):
    """One Dormand-Prince step of Eq. (6) (beyond the paper, which uses Euler).
    Stages at plain (not renormalised) states Y_i = M + dt sum_j a_ij k_j; the
    fifth-order state M + dt sum_i b_i k_i is renormalised to |M| = Ms; the
    seventh stage k7 is evaluated there and serves as k1 of the next step
    (first same as last).  The error estimate is
      err = max over cells |dt sum_i e_i k_i| / Ms.
    k1 = f(M) is passed in.  Returns (M_new, err, k7)."""
    f = lambda X: _rhs(X, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L)
    ks = [k1]
    for i in range(1, 6):
        Y = M + dt * sum(DP_A[i][j] * ks[j] for j in range(i))
        ks.append(f(Y))
    Y5 = M + dt * sum(DP_B[j] * ks[j] for j in range(6))
    Mn = Y5 * (Ms / np.sqrt(np.sum(Y5 * Y5, axis=0)))
    k7 = f(Mn)
    ks.append(k7)
    D = dt * sum(DP_E[j] * ks[j] for j in range(7))
    err = float(np.max(np.sqrt(np.sum(D * D, axis=0)))) / Ms
    return Mn, err, k7


# Step-size controller of the adaptive run: a step is accepted when
# err <= tol; the next step is h * clamp(0.9 (tol / err)^(1/5), 0.2, 5), with
# no growth right after a rejection; the last step is shortened to end on
# t_span.
DP_SAFETY, DP_FMIN, DP_FMAX = 0.9, 0.2, 5.0


def dp_next_factor(err, tol, after_reject):
    fac = DP_FMAX if err <= 0.0 else DP_SAFETY * (tol / err) ** 0.2
    fac = min(DP_FMAX, max(DP_FMIN, fac))
    return min(fac, 1.0) if after_reject else fac


def run_dopri5(M, t_span, dt0, tol, max_steps, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L):
    """Adaptive Dormand-Prince integration of Eq. (6) over t_span.  Returns
    (M, dt_next, (accepted, rejected, field evaluations, time covered))."""
    f = lambda X: _rhs(X, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L)
    k1 = f(M)
    t, dt, acc, rej, nev = 0.0, dt0, 0, 0, 1
    after_reject = False
    while t_span - t > 1e-12 * t_span and acc + rej < max_steps:
        h = min(dt, t_span - t)
        Mn, err, k7 = dopri5_step(M, k1, h, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L)
        nev += 6
        if err <= tol:
            t += h
            M, k1 = Mn, k7
            acc += 1
            dt = h * dp_next_factor(err, tol, after_reject)
            after_reject = False
        else:
            rej += 1
            dt = h * dp_next_factor(err, tol, True)
            after_reject = True
    return M, dt, (acc, rej, nev, t)


def run_euler(M, nsteps, dt, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L):
    for _ in range(nsteps):
        M, _ = euler_step(M, dt, cell, Ms, A, Ku, alpha, gamma, H_ext, Kt, L)
    return M


def energy_terms(M, H_demag, cell, Ms, A, Ku, H_ext):
    """Eq. (1) integrated over the sample, in joules:
    (total, exchange, anisotropy, demag, Zeeman).

    Exchange is the link sum A V sum_links |m_i - m_j|^2 / delta^2 (m =
    M/Ms), the discrete form of A (grad m)^2 that matches Eq. (4) with
    Neumann boundaries."""
    dx, dy, dz = cell
    V = dx * dy * dz
    m = M / Ms
    ex = 0.0
    for axis, d in ((3, dx), (2, dy), (1, dz)):
        diff = np.diff(m, axis=axis)
        ex += np.sum(diff * diff) / (d * d)
    ex *= A * V
    an = Ku * V * np.sum(M[1] ** 2 + M[2] ** 2) / (Ms * Ms)
    de = -0.5 * MU0 * V * np.sum(H_demag * M)
    ze = -MU0 * V * np.sum(np.asarray(H_ext, np.float64).reshape(3, 1, 1, 1) * M)
    return np.array([ex + an + de + ze, ex, an, de, ze])


def macrospin_closed_form(theta0, phi0, H, alpha, gamma, t):
    """Exact solution of Eq. (6) for one moment in a static field H along +z
    (no other torque): the polar angle obeys
    tan(theta/2) = tan(theta0/2) exp(-alpha gamma H t / (1 + alpha^2)) and the
    azimuth advances as phi0 + gamma H t / (1 + alpha^2)."""
    w = gamma * H / (1.0 + alpha * alpha)
    theta = 2.0 * np.arctan(np.tan(theta0 / 2.0) * np.exp(-alpha * w * t))
    phi = phi0 + w * t
    return theta, phi
