"""Klein-step transmission for the smooth step V(x) = V0/2 [1 + tanh(x/L)] (Sec. 5.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Two independent routes:
  * ``transmission_closed_form``: Eq. trans_co, read with k = +(1/c) sqrt((E-V0)^2 - m^2c^4),
    k' = -(1/c) sqrt(E^2 - m^2c^4) as printed and V0/c in the sinh arguments.  It applies in
    the Klein regime E < V0 - mc^2; inside the gap |E - V0| < mc^2 a plane wave is not
    transmitted (T = 0).
  * ``transmission_ode``: the stationary 1-D Dirac equation H psi = E psi with
    H = c alpha_x p + beta m c^2 + V(x) (Eq. hamiltonian, A = 0), restricted to the
    (psi1, psi4) pair that alpha_x couples, integrated across the step with fixed-step RK4
    from a purely transmitted wave on the right, then split into incident and reflected
    waves on the left.  T and R are ratios of the currents j = c psi^dag alpha_x psi.
Atomic units: m = 1, c = 137.0359895 (Sec. 5).
"""
from __future__ import annotations

import numpy as np

C_AU = 137.0359895


def energy(k0: float, m: float = 1.0, c: float = C_AU) -> float:
    """E_k = sqrt(k0^2 c^2 + m^2 c^4)."""
    return float(np.sqrt(k0 * k0 * c * c + m * m * c ** 4))


def transmission_closed_form(k0: float, V0: float, L: float, m: float = 1.0, c: float = C_AU) -> float:
    """Eq. trans_co for an incident momentum k0 (a.u.)."""
    E = energy(k0, m, c)
    if abs(E - V0) < m * c * c:
        return 0.0  # evanescent inside the step: no propagating transmitted wave
    if E > V0 + m * c * c:
        raise ValueError("over-barrier energy: Eq. trans_co is read for the Klein regime only; use transmission_ode")
    k = np.sqrt((E - V0) ** 2 - m * m * c ** 4) / c
    kp = -np.sqrt(E * E - m * m * c ** 4) / c
    num = np.sinh(np.pi * k * L) * np.sinh(np.pi * kp * L)
    den = np.sinh(np.pi * (V0 / c + k + kp) * L / 2) * np.sinh(np.pi * (V0 / c - k - kp) * L / 2)
    return float(-num / den)


def transmission_sharp_step(k0: float, V0: float, m: float = 1.0, c: float = C_AU) -> float:
    """L -> 0 limit: continuity of (psi1, psi4) at a sharp step gives T = 4 kappa / (1 + kappa)^2,
    kappa = q (E + mc^2) / ((E - V0 + mc^2) p), p = k0, q the transmitted momentum whose current is
    positive."""
    E = energy(k0, m, c)
    if abs(E - V0) < m * c * c:
        return 0.0
    q = np.sqrt((E - V0) ** 2 - m * m * c ** 4) / c
    if E - V0 + m * c * c < 0:
        q = -q  # hole-like branch: positive current needs negative momentum
    kappa = q * (E + m * c * c) / ((E - V0 + m * c * c) * k0)
    return float(4 * kappa / (1 + kappa) ** 2)


def _rhs(E, V, m, c):
    def f(x, y):
        v = V(x)
        return np.array([1j / c * (E - v + m * c * c) * y[1], 1j / c * (E - v - m * c * c) * y[0]])
    return f


def transmission_ode(k0: float, V0: float, L: float, m: float = 1.0, c: float = C_AU,
                     half_width: float | None = None, nstep: int = 40000):
    """(T, R) from fixed-step RK4 of d/dx (psi1, psi4) = (i/c) ((E-V+mc^2) psi4, (E-V-mc^2) psi1)."""
    E = energy(k0, m, c)
    p = k0
    if half_width is None:
        half_width = 40.0 * L
    V = lambda x: 0.5 * V0 * (1.0 + np.tanh(x / L))
    xr, xl = half_width, -half_width
    v_r = V(xr)
    if (E - v_r) ** 2 <= (m * c * c) ** 2:
        return 0.0, 1.0
    q = np.sqrt((E - v_r) ** 2 - (m * c * c) ** 2) / c
    r_t = c * q / (E - v_r + m * c * c)
    if r_t < 0:  # current 2 c r_t must be positive for the transmitted wave
        q = -q
        r_t = -r_t
    y = np.array([1.0 + 0j, r_t + 0j]) * np.exp(1j * q * xr)
    f = _rhs(E, V, m, c)
    h = (xl - xr) / nstep
    x = xr
    for _ in range(nstep):
        k1 = f(x, y)
        k2 = f(x + h / 2, y + h / 2 * k1)
        k3 = f(x + h / 2, y + h / 2 * k2)
        k4 = f(x + h, y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        x = x + h
    v_l = V(xl)
    pl = np.sqrt((E - v_l) ** 2 - (m * c * c) ** 2) / c
    rp = c * pl / (E - v_l + m * c * c)
    # y = A (1, rp) e^{i pl x} + B (1, -rp) e^{-i pl x}
    a_e = 0.5 * (y[0] + y[1] / rp)
    b_e = 0.5 * (y[0] - y[1] / rp)
    A = a_e * np.exp(-1j * pl * xl)
    B = b_e * np.exp(1j * pl * xl)
    j_inc = 2 * c * rp * abs(A) ** 2
    j_ref = 2 * c * rp * abs(B) ** 2
    j_tr = 2 * c * r_t
    return float(j_tr / j_inc), float(j_ref / j_inc)


def packet_averaged_transmission(k0: float, width: float, V0: float, L: float, m: float = 1.0,
                                 c: float = C_AU, npts: int = 201) -> float:
    """Closed form averaged over the momentum density |phi(p)|^2 ~ exp(-2 width^2 (p-k0)^2) of a
    Gaussian packet exp(-(x-x0)^2/(4 width^2)) (one-dimensional reading)."""
    sig = 1.0 / (2.0 * width)
    ps = k0 + sig * np.linspace(-6, 6, npts)
    w = np.exp(-0.5 * ((ps - k0) / sig) ** 2)
    t = np.array([transmission_closed_form(p, V0, L, m, c) for p in ps])
    return float((w * t).sum() / w.sum())
