"""Seeded synthetic inputs for the Dirac stepper: initial spinors, potentials and
run-parameter draws.

This module holds none of the scheme's arithmetic (no sweep, no phase, no
observable); it only builds the inputs that both the CUDA path and the CPU
oracle consume.  It imports numpy only.

Units are atomic units (Sec. 5): m = 1, c = 137.0359895, hbar = |e| = 1.
The cell edge defaults to dx = 10/8192 a.u. (the paper's 2-D mesh spacing), so
that dt = dx/c = 8.9e-6 a.u. satisfies the time-step bound of Sec. 2.5.
State arrays are complex128 of shape (nz, ny, nx, 4) (ny = 1 for the x-z plane).
"""
from __future__ import annotations

import dataclasses

import numpy as np

C_AU = 137.0359895
M_E = 1.0
DX_DEFAULT = 10.0 / 8192.0
SEED = 20111107


def cell_centres(n: int, dx: float, x_min: float) -> np.ndarray:
    """x_min + (i + 1/2) dx, i = 0..n-1 (Sec. 2.3)."""
    return x_min + (np.arange(n) + 0.5) * dx


def normalise(psi: np.ndarray, dx: float, ndim: int) -> np.ndarray:
    """Scale so that sum |psi|^2 dx^ndim = 1."""
    rho = (psi.real ** 2 + psi.imag ** 2).sum()
    return psi / np.sqrt(rho * dx ** ndim)


def spinor_C(k0: float, m: float = M_E, c: float = C_AU) -> float:
    """C = c k0 / (mc^2 + sqrt(m^2 c^4 + c^2 k0^2)) of the travelling packet (Sec. 5.1.4)."""
    return c * k0 / (m * c * c + np.sqrt(m * m * c ** 4 + c * c * k0 * k0))


def gaussian_packet(nx: int, nz: int, dx: float, x_min: float, z_min: float, x0: float, z0: float,
                    width: float, k0: float, m: float = M_E, c: float = C_AU, ny: int = 1,
                    y_min: float = 0.0, y0: float = 0.0) -> np.ndarray:
    """N [1, 0, 0, C] e^{i k0 x} exp(-|r - r0|^2 / (4 width^2)) (Sec. 5.1.4 and 5.2.2), normalised.

    With ny > 1 the Gaussian also extends along y (3-D)."""
    x = cell_centres(nx, dx, x_min)
    z = cell_centres(nz, dx, z_min)
    gx = np.exp(-((x - x0) ** 2) / (4 * width ** 2)) * np.exp(1j * k0 * x)
    gz = np.exp(-((z - z0) ** 2) / (4 * width ** 2))
    if ny > 1:
        y = cell_centres(ny, dx, y_min)
        gy = np.exp(-((y - y0) ** 2) / (4 * width ** 2))
    else:
        gy = np.ones(1)
    g = gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    spin = np.array([1.0, 0.0, 0.0, spinor_C(k0, m, c)], dtype=np.complex128)
    psi = g[..., None] * spin
    return normalise(psi.astype(np.complex128), dx, 3 if ny > 1 else 2)


def positive_energy_packet_2d(nx: int, nz: int, dx: float, width: float, k0: float,
                              m: float = M_E, c: float = C_AU) -> np.ndarray:
    """Gaussian centred in the box, projected per Fourier mode of the periodic box onto the
    positive-energy eigenspace of the free Hamiltonian c(alpha_x p_x + alpha_z p_z) + beta mc^2
    (projector (1 + H(p)/E(p))/2), then normalised.  The box is [-nx dx/2, nx dx/2) x [-nz dx/2, nz dx/2)."""
    psi = gaussian_packet(nx, nz, dx, -nx * dx / 2, -nz * dx / 2, 0.0, 0.0, width, k0, m, c)[:, 0]
    px = 2 * np.pi * np.fft.fftfreq(nx, d=dx)
    pz = 2 * np.pi * np.fft.fftfreq(nz, d=dx)
    PX, PZ = np.meshgrid(px, pz)  # (nz, nx)
    ax, az, beta = _dirac_alpha_x(), _dirac_alpha_z(), _dirac_beta()
    H = c * (PX[..., None, None] * ax + PZ[..., None, None] * az) + m * c * c * beta
    E = np.sqrt((c * PX) ** 2 + (c * PZ) ** 2 + (m * c * c) ** 2)
    P = 0.5 * (np.eye(4) + H / E[..., None, None])
    hat = np.fft.fft2(psi, axes=(0, 1))
    hat = np.einsum("zxab,zxb->zxa", P, hat)
    out = np.fft.ifft2(hat, axes=(0, 1))[:, None]
    return normalise(out, dx, 2)


def _dirac_beta():
    return np.diag([1.0, 1.0, -1.0, -1.0]).astype(np.complex128)


def _dirac_alpha_x():
    a = np.zeros((4, 4), np.complex128)
    a[0, 3] = a[1, 2] = a[2, 1] = a[3, 0] = 1.0
    return a


def _dirac_alpha_z():
    a = np.zeros((4, 4), np.complex128)
    a[0, 2] = 1.0
    a[1, 3] = -1.0
    a[2, 0] = 1.0
    a[3, 1] = -1.0
    return a


def tanh_step(nx: int, dx: float, x_min: float, x_s: float, V0: float, L: float) -> np.ndarray:
    """V(x) = V0/2 [1 + tanh((x - x_s)/L)] at the x cell centres (Sec. 5.2.1), one value per column."""
    x = cell_centres(nx, dx, x_min)
    return 0.5 * V0 * (1.0 + np.tanh((x - x_s) / L))


def soft_coulomb_3d(n: int, dx: float, Z: float, a: float) -> np.ndarray:
    """V = -Z / sqrt(r^2 + a^2) on an n^3 grid centred on the box centre, shape (n, n, n) [z][y][x]."""
    x = cell_centres(n, dx, -n * dx / 2)
    r2 = x[None, None, :] ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2
    return -Z / np.sqrt(r2 + a * a)


def random_state(nz: int, ny: int, nx: int, seed: int) -> np.ndarray:
    """Complex Gaussian noise, unit-normalised with dx = 1 (for parity on unstructured inputs)."""
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal((nz, ny, nx, 4)) + 1j * rng.standard_normal((nz, ny, nx, 4))
    return psi / np.sqrt((np.abs(psi) ** 2).sum())


def absorber_mask(nx: int, cells: int, eta: float) -> np.ndarray:
    """Per-x-column damping factors of an absorbing layer of `cells` columns at each x edge:
    a = exp(-eta s^2) with s = distance into the layer / cells (1/cells at its inner column, 1 at the edge),
    1 elsewhere.  Applied with the phase every step (not part of the paper's scheme)."""
    if cells <= 0:
        return np.ones(nx)
    i = np.arange(nx)
    s_left = np.clip((cells - i) / cells, 0.0, 1.0)
    s_right = np.clip((i - (nx - cells) + 1) / cells, 0.0, 1.0)
    s = np.maximum(s_left, s_right)
    return np.exp(-eta * s * s)


def laser_A_tilde(nsteps: int, dt: float, A0: float, omega: float, ncycles: float, pol=(1.0, 0.0, 0.0),
                  charge: float = -1.0, step0: int = 0) -> np.ndarray:
    """Per-step integrals At_n = e * int_{t_n}^{t_{n+1}} A(t) dt (Eq. field_dis1) of a uniform (dipole)
    laser pulse A(t) = A0 sin^2(pi t / tau) sin(omega t) pol for 0 <= t <= tau = 2 pi ncycles / omega, zero
    after, with t_n = (step0 + n) dt.  The integral is analytic: with W = 2 pi / tau,
    sin^2(W t / 2) sin(omega t) = sin(omega t)/2 - [sin((omega + W) t) + sin((omega - W) t)]/4.
    Returns an (nsteps, 3) array (input data: the scheme itself never integrates the field)."""
    tau = 2.0 * np.pi * ncycles / omega
    Wf = 2.0 * np.pi / tau

    def F(t):
        t = np.clip(t, 0.0, tau)
        out = -np.cos(omega * t) / (2.0 * omega)
        for w in (omega + Wf, omega - Wf):
            out = out + (np.cos(w * t) / (4.0 * w) if w != 0.0 else -t * 0.0)
        return out

    t = (step0 + np.arange(nsteps + 1)) * dt
    integ = F(t[1:]) - F(t[:-1])
    return charge * A0 * integ[:, None] * np.asarray(pol, dtype=np.float64)[None, :]


ABSORB_CELLS = 64      # absorbing layer at each x edge of an ensemble run
ABSORB_ETA = 0.1
BEYOND_STEP = 128      # cells kept between the step face and the right absorbing layer


@dataclasses.dataclass
class KleinRun:
    """One 2-D Klein-step scattering run on a square grid of `side` cells."""
    side: int
    V0: float       # step height, a.u.
    p0: float       # packet momentum along x, a.u.
    width: float    # Gaussian width Delta, a.u.
    nsteps: int
    dx: float = DX_DEFAULT
    L: float = 4 * DX_DEFAULT
    face: int = -1  # flux face index (the step is centred on it)
    absorb: int = 0  # absorbing-layer columns at each x edge (0: none)
    eta: float = ABSORB_ETA

    def geometry(self):
        """(x_min, z_min, x_s, x0): the step sits on face `face` (x = 0), the packet 4 widths left of it."""
        face = self.face if self.face >= 0 else (5 * self.side) // 8
        x_min = -face * self.dx
        z_min = -(self.side // 2) * self.dx
        return x_min, z_min, 0.0, -4.0 * self.width, face

    def state(self, m: float = M_E, c: float = C_AU) -> np.ndarray:
        """The Gaussian packet (normalised over the grid), zero inside the absorbing layers."""
        x_min, z_min, x_s, x0, _ = self.geometry()
        psi = gaussian_packet(self.side, self.side, self.dx, x_min, z_min, x0, 0.0, self.width, self.p0, m, c)
        if self.absorb > 0:
            psi[:, :, :self.absorb, :] = 0
            psi[:, :, self.side - self.absorb:, :] = 0
        return psi

    def mask(self) -> np.ndarray:
        return absorber_mask(self.side, self.absorb, self.eta)

    def potential(self) -> np.ndarray:
        x_min, _, x_s, _, _ = self.geometry()
        return tanh_step(self.side, self.dx, x_min, x_s, self.V0, self.L)

    def as_batch_fields(self) -> dict:
        """Fields of the library's dirac_klein_run (packet centre relative to the step at x = 0)."""
        _, _, _, x0, face = self.geometry()
        return {"side": self.side, "face": face, "nsteps": self.nsteps, "V0": self.V0, "L": self.L,
                "p0": self.p0, "width": self.width, "x0": x0, "absorb": self.absorb, "eta": self.eta}


def klein_config_2d(seed: int = SEED, side: int = 2048, nsteps: int = 4000, m: float = M_E, c: float = C_AU) -> KleinRun:
    """2-D Klein step, FP64 workload: 2048^2 cells, V0 = 2.5 mc^2, L = 4 dx, width 100 dx,
    p0 ~ U[0.2, 1.0] mc drawn from numpy PCG64(seed), 4000 steps, step face at 5/8 of the x extent."""
    rng = np.random.default_rng(seed)
    p0 = rng.uniform(0.2, 1.0) * m * c
    dx = DX_DEFAULT
    return KleinRun(side=side, V0=2.5 * m * c * c, p0=p0, width=100 * dx, nsteps=nsteps, dx=dx, L=4 * dx)


ALLOWED_SIDES = (256, 384, 512, 768, 1024)


def klein_ensemble(nruns: int = 512, seed: int = SEED + 1, m: float = M_E, c: float = C_AU):
    """Batched ensemble draws: side U{256..1024}, V0 ~ U[0.5, 3.0] mc^2, p0 ~ U[0.2, 1.0] mc,
    width ~ U[40, 150] dx.  Each run has 64-column absorbing layers at both x edges (the zero boundary
    reflects part of a massive wave, and a reflection that comes back across the face corrupts the
    transmitted fraction).  A drawn side smaller than 8 width + 264 cells is raised to the smallest allowed
    side that holds the packet clear of the left layer and 128 cells plus the right layer beyond the step
    (1024 at most; wider packets are cut at the left layer); the step face sits 8 widths + 8 cells right of
    the left layer but at least 128 + 64 cells from the right edge, the packet 4 widths left of the face;
    the step count is the time for the packet centre to travel 8 widths at the group velocity p0 c^2 / E
    plus 200, clamped to [2000, 6000].  Returns (runs, log) where log lists every deviation from the drawn
    values."""
    rng = np.random.default_rng(seed)
    dx = DX_DEFAULT
    runs, log = [], []
    for r in range(nruns):
        side = int(rng.choice(ALLOWED_SIDES))
        V0 = rng.uniform(0.5, 3.0) * m * c * c
        p0 = rng.uniform(0.2, 1.0) * m * c
        w_cells = rng.uniform(40, 150)
        need = 8 * w_cells + 8 + BEYOND_STEP + 2 * ABSORB_CELLS
        if side < need:
            bigger = [s for s in ALLOWED_SIDES if s >= need]
            new = bigger[0] if bigger else ALLOWED_SIDES[-1]
            log.append((r, "side", side, new))
            side = new
        E = np.sqrt(p0 * p0 * c * c + m * m * c ** 4)
        vg_over_c = p0 * c / E
        nsteps = int(np.clip(np.ceil(8 * w_cells / vg_over_c) + 200, 2000, 6000))
        face = min(int(np.ceil(8 * w_cells)) + 8 + ABSORB_CELLS, side - BEYOND_STEP - ABSORB_CELLS)
        runs.append(KleinRun(side=side, V0=V0, p0=p0, width=w_cells * dx, nsteps=nsteps, dx=dx, L=4 * dx,
                             face=face, absorb=ABSORB_CELLS, eta=ABSORB_ETA))
    return runs, log


DRAWN_SIDES_ABSORB = 16   # absorbing columns at each x edge in the drawn-sides ensemble
DRAWN_SIDES_BEYOND = 32   # cells between the step and the right layer in the drawn-sides ensemble


def klein_ensemble_drawn_sides(nruns: int = 512, seed: int = SEED + 7, m: float = M_E, c: float = C_AU):
    """An ensemble whose runs keep their drawn sides U{256, 384, 512, 768, 1024}, for measuring how the persistent
    kernel's task queue balances truly uneven grids (up to 16x in cells and 3x in steps).  V0, p0 and the width
    are drawn as in klein_ensemble; the width is then capped so that the packet (4 widths left of the step, 4
    widths of tail) fits the drawn side with 16-column absorbing layers and 32 cells beyond the step, so the
    narrow grids carry narrow packets.  The transmissions of these runs are not the configuration's physics (the
    short region beyond the step lets evanescent waves reach the layer); only their cost and balance matter.
    Returns (runs, log) with every capped width logged."""
    rng = np.random.default_rng(seed)
    dx = DX_DEFAULT
    runs, log = [], []
    for r in range(nruns):
        side = int(rng.choice(ALLOWED_SIDES))
        V0 = rng.uniform(0.5, 3.0) * m * c * c
        p0 = rng.uniform(0.2, 1.0) * m * c
        w_cells = rng.uniform(40, 150)
        cap = (side - 8 - DRAWN_SIDES_BEYOND - 2 * DRAWN_SIDES_ABSORB) / 8.0
        if w_cells > cap:
            log.append((r, "width", w_cells, cap))
            w_cells = cap
        E = np.sqrt(p0 * p0 * c * c + m * m * c ** 4)
        nsteps = int(np.clip(np.ceil(8 * w_cells / (p0 * c / E)) + 200, 2000, 6000))
        face = min(int(np.ceil(8 * w_cells)) + 8 + DRAWN_SIDES_ABSORB, side - DRAWN_SIDES_BEYOND - DRAWN_SIDES_ABSORB)
        runs.append(KleinRun(side=side, V0=V0, p0=p0, width=w_cells * dx, nsteps=nsteps, dx=dx, L=4 * dx,
                             face=face, absorb=DRAWN_SIDES_ABSORB, eta=ABSORB_ETA))
    return runs, log


def packet_mass_right_of_step(width_cells: float = 1.0) -> float:
    """Fraction of a Gaussian packet |psi|^2 ~ exp(-(x - x0)^2 / (2 width^2)) centred 4 widths left of the step
    that already lies right of it: erfc(4 / sqrt 2) / 2 (independent of the width).  The net flux through the
    face, the ensembles' T, can go below zero by at most this much: that part can only flow back."""
    from math import erfc, sqrt
    return 0.5 * erfc(4.0 / sqrt(2.0))
