"""Independent linear-algebra statements of the scheme used to pin the oracle.

Nothing here is taken from the oracle: the Dirac matrices are built from the
Pauli matrices (Eq. dirac_mat), the sweeps as explicit 4N x 4N matrices
(Eqs. sol_dis_1-3), the phase from the exponential identity for Dirac matrices
(Sec. 2.3, e^{i(beta F + alpha.F)} = cos|F| + i (beta F + alpha.F)/|F| sin|F|),
and the Fourier statements from numpy's FFT.
"""
from __future__ import annotations

import numpy as np

SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)
I4 = np.eye(4, dtype=np.complex128)

BETA = np.kron(np.diag([1.0, -1.0]), I2).astype(np.complex128)
ALPHA = [np.kron(SX, s) for s in (SX, SY, SZ)]  # [[0, s], [s, 0]]


def sweep_matrix(n, axis: int, periodic: bool, shift: int = 1) -> np.ndarray:
    """Dense matrix of one directional sweep on a grid n = (nx, ny, nz), state flattened as
    ((k*ny + j)*nx + i)*4 + c; neighbours at +-shift cells (c dt = shift * dx)."""
    nx, ny, nz = n
    N = nx * ny * nz
    M = np.zeros((4 * N, 4 * N), dtype=np.complex128)
    Pp = 0.5 * (I4 + ALPHA[axis])
    Pm = 0.5 * (I4 - ALPHA[axis])
    d = [0, 0, 0]
    d[axis] = shift

    def idx(i, j, k):
        if periodic:
            i, j, k = i % nx, j % ny, k % nz
        elif not (0 <= i < nx and 0 <= j < ny and 0 <= k < nz):
            return None
        return (k * ny + j) * nx + i

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                o = idx(i, j, k)
                lft = idx(i - d[0], j - d[1], k - d[2])
                rgt = idx(i + d[0], j + d[1], k + d[2])
                if lft is not None:
                    M[4 * o:4 * o + 4, 4 * lft:4 * lft + 4] += Pp
                if rgt is not None:
                    M[4 * o:4 * o + 4, 4 * rgt:4 * rgt + 4] += Pm
    return M


def dirac_exp(F: float, Fvec) -> np.ndarray:
    """e^{i(beta F + alpha.F)} from the closed form of Sec. 2.3."""
    Fvec = np.asarray(Fvec, dtype=float)
    mag = np.sqrt(F * F + Fvec @ Fvec)
    G = F * BETA + sum(f * a for f, a in zip(Fvec, ALPHA))
    if mag == 0:
        return I4.copy()
    return np.cos(mag) * I4 + 1j * G / mag * np.sin(mag)


def phase_matrix(n, m, c, dt, Vcell) -> np.ndarray:
    """Block-diagonal exp(-i beta m c^2 dt) exp(-i V dt) per cell (Eq. sol_dis_4, A = 0);
    Vcell is one value per cell in flattened cell order."""
    nx, ny, nz = n
    N = nx * ny * nz
    M = np.zeros((4 * N, 4 * N), dtype=np.complex128)
    U = dirac_exp(-m * c * c * dt, [0.0, 0.0, 0.0])
    for o in range(N):
        M[4 * o:4 * o + 4, 4 * o:4 * o + 4] = U * np.exp(-1j * Vcell[o] * dt)
    return M


def amplification_2d(kx, kz, nx, nz, mu):
    """Per-mode one-step matrix of the periodic 2-D scheme: e^{-i beta mu} e^{-i alpha_z th_z} e^{-i alpha_x th_x},
    th = 2 pi k / N (Eq. sol_dis and its 3-D counterpart in Sec. 3.2)."""
    thx = 2 * np.pi * kx / nx
    thz = 2 * np.pi * kz / nz
    Ux = np.cos(thx)[..., None, None] * I4 - 1j * np.sin(thx)[..., None, None] * ALPHA[0]
    Uz = np.cos(thz)[..., None, None] * I4 - 1j * np.sin(thz)[..., None, None] * ALPHA[2]
    Ub = np.cos(mu) * I4 - 1j * np.sin(mu) * BETA
    return Ub @ Uz @ Ux


def dft_exact_evolution_2d(psi0: np.ndarray, nsteps: int, mu: float, shift: int = 1) -> np.ndarray:
    """psi after nsteps of the periodic V = 0 scheme, computed mode by mode in Fourier space.
    psi0 has shape (nz, 1, nx, 4).  With characteristic shift K a sweep moves by K cells: th = 2 pi k K / N."""
    nz, _, nx, _ = psi0.shape
    hat = np.fft.fft2(psi0[:, 0], axes=(0, 1))
    KX, KZ = np.meshgrid(np.arange(nx), np.arange(nz))
    U = amplification_2d(shift * KX, shift * KZ, nx, nz, mu)
    Un = np.linalg.matrix_power(U, nsteps)
    hat = np.einsum("zxab,zxb->zxa", Un, hat)
    return np.fft.ifft2(hat, axes=(0, 1))[:, None]


def continuum_evolution_2d(psi0: np.ndarray, dx: float, t: float, m: float, c: float) -> np.ndarray:
    """Exact free evolution e^{-i (c alpha.p + beta m c^2) t} in Fourier space (App. B), sampled on the
    periodic grid: p = 2 pi fftfreq(N, dx) along x and z."""
    nz, _, nx, _ = psi0.shape
    px = 2 * np.pi * np.fft.fftfreq(nx, d=dx)
    pz = 2 * np.pi * np.fft.fftfreq(nz, d=dx)
    PX, PZ = np.meshgrid(px, pz)
    E = np.sqrt((c * PX) ** 2 + (c * PZ) ** 2 + (m * c * c) ** 2)
    H = c * (PX[..., None, None] * ALPHA[0] + PZ[..., None, None] * ALPHA[2]) + m * c * c * BETA
    sinE = np.where(E > 0, np.sin(E * t) / np.where(E > 0, E, 1.0), t)  # sin(Et)/E -> t at E = 0 (m = 0, p = 0)
    U = np.cos(E * t)[..., None, None] * I4 - 1j * sinE[..., None, None] * H
    hat = np.fft.fft2(psi0[:, 0], axes=(0, 1))
    hat = np.einsum("zxab,zxb->zxa", U, hat)
    return np.fft.ifft2(hat, axes=(0, 1))[:, None]


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def phase_matrix_A_cell(m, c, dt, v, At) -> np.ndarray:
    """exp(-i dt (beta m c^2 + v - alpha.(At/dt))) for one cell, by scipy's matrix exponential of the 4x4
    generator (Eq. sol_dis_4 before the closed form of Sec. 2.3 is applied)."""
    from scipy.linalg import expm
    G = -1j * (m * c * c * dt) * BETA - 1j * v * dt * I4 + 1j * sum(a * M for a, M in zip(At, ALPHA))
    return expm(G)


def dft_exact_evolution_2d_A(psi0: np.ndarray, mu: float, At_steps, m_c2_dt=None) -> np.ndarray:
    """psi after len(At_steps) periodic V = 0 steps with a uniform vector potential: mode by mode
    U_n = exp(-i beta mu + i alpha.At_n) e^{-i alpha_z th_z} e^{-i alpha_x th_x} (matrix exponential by scipy)."""
    from scipy.linalg import expm
    nz, _, nx, _ = psi0.shape
    hat = np.fft.fft2(psi0[:, 0], axes=(0, 1))
    KX, KZ = np.meshgrid(np.arange(nx), np.arange(nz))
    S = amplification_2d(KX, KZ, nx, nz, 0.0)  # sweeps only (mu = 0: the mass phase is the identity)
    for At in At_steps:
        UA = expm(-1j * mu * BETA + 1j * sum(a * M for a, M in zip(At, ALPHA)))
        hat = np.einsum("ab,zxbc,zxc->zxa", UA, S, hat)
    return np.fft.ifft2(hat, axes=(0, 1))[:, None]


def continuum_evolution_3d(psi0: np.ndarray, dx: float, t: float, m: float, c: float) -> np.ndarray:
    """Exact free evolution e^{-i (c alpha.p + beta m c^2) t} in Fourier space on the periodic 3-D grid
    (psi0 shape (nz, ny, nx, 4))."""
    nz, ny, nx, _ = psi0.shape
    px = 2 * np.pi * np.fft.fftfreq(nx, d=dx)
    py = 2 * np.pi * np.fft.fftfreq(ny, d=dx)
    pz = 2 * np.pi * np.fft.fftfreq(nz, d=dx)
    PZ, PY, PX = np.meshgrid(pz, py, px, indexing="ij")
    E = np.sqrt((c * PX) ** 2 + (c * PY) ** 2 + (c * PZ) ** 2 + (m * c * c) ** 2)
    H = c * (PX[..., None, None] * ALPHA[0] + PY[..., None, None] * ALPHA[1] + PZ[..., None, None] * ALPHA[2]) \
        + m * c * c * BETA
    sinE = np.where(E > 0, np.sin(E * t) / np.where(E > 0, E, 1.0), t)
    U = np.cos(E * t)[..., None, None] * I4 - 1j * sinE[..., None, None] * H
    hat = np.fft.fftn(psi0, axes=(0, 1, 2))
    hat = np.einsum("zyxab,zyxb->zyxa", U, hat)
    return np.fft.ifftn(hat, axes=(0, 1, 2))


def phase_matrix_field(n, m, c, dt, vt_cells, At_cells) -> np.ndarray:
    """Block-diagonal exp(-i beta m c^2 dt - i V~(i) + i alpha.At(i)) per cell (scipy's matrix exponential of
    each cell's 4x4 generator); vt_cells: V~ per cell, At_cells: (ncells, 3), cells in flattened order."""
    from scipy.linalg import expm
    nx, ny, nz = n
    N = nx * ny * nz
    M = np.zeros((4 * N, 4 * N), dtype=np.complex128)
    for o in range(N):
        G = -1j * (m * c * c * dt) * BETA - 1j * vt_cells[o] * I4 + 1j * sum(a * Al for a, Al in zip(At_cells[o], ALPHA))
        M[4 * o:4 * o + 4, 4 * o:4 * o + 4] = expm(G)
    return M
