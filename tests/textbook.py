"""Textbook forms used to pin the oracle (written independently of oracle/).

  D2Q9 velocity set and equilibrium weights t = (4/9, 1/9 x4, 1/36 x4).
  Second-order equilibrium f_eq = t rho [1 + 3 e.v + 9/2 (e.v)^2 - 3/2 v^2].
  Lallemand-Luo moment basis built from its polynomial definitions
    (1, -4 + 3|e|^2, 4 - 21/2 |e|^2 + 9/2 |e|^4, e_x, (-5 + 3|e|^2) e_x, e_y,
     (-5 + 3|e|^2) e_y, e_x^2 - e_y^2, e_x e_y).
  Guo et al. (2002) forcing in velocity space with c_s^2 = 1/3:
    S_a = t_a [3 (e_a - v).F + 9 (e_a.v)(e_a.F)].
  A velocity-space MRT update (Eq. 1 with Lambda_bar = M^-1 Lambda M) and a BGK update
  with Guo forcing, both on periodic numpy arrays (Q, ny, nx).
"""
import numpy as np

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
T_W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W_FORCE = np.array([0.0] + [1 / 3] * 4 + [1 / 12] * 4)


def moment_basis():
    e2 = EX ** 2 + EY ** 2
    rows = [np.ones(9), -4 + 3 * e2, 4 - 10.5 * e2 + 4.5 * e2 ** 2, EX, (-5 + 3 * e2) * EX,
            EY, (-5 + 3 * e2) * EY, EX ** 2 - EY ** 2, EX * EY]
    return np.array(rows, dtype=float)


def feq(rho, ux, uy):
    rho, ux, uy = np.broadcast_arrays(np.asarray(rho, float), ux, uy)
    eu = EX.reshape((9,) + (1,) * rho.ndim) * ux + EY.reshape((9,) + (1,) * rho.ndim) * uy
    u2 = ux * ux + uy * uy
    t = T_W.reshape((9,) + (1,) * rho.ndim)
    return t * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * u2)


def guo_source(ux, uy, Fx, Fy):
    nd = np.ndim(ux)
    ex = EX.reshape((9,) + (1,) * nd)
    ey = EY.reshape((9,) + (1,) * nd)
    t = T_W.reshape((9,) + (1,) * nd)
    eu = ex * ux + ey * uy
    eF = ex * Fx + ey * Fy
    return t * (3 * ((ex - ux) * Fx + (ey - uy) * Fy) + 9 * eu * eF)


def stream_periodic(fs):
    out = np.empty_like(fs)
    for a in range(9):
        out[a] = np.roll(np.roll(fs[a], EY[a], axis=0), EX[a], axis=1)
    return out


def psi_F(rho, psi_of_rho, G):
    """psi per node and the force of Eq. 7 on a periodic grid (numpy rolls)."""
    psi = np.vectorize(psi_of_rho)(rho)
    Sx = np.zeros_like(rho)
    Sy = np.zeros_like(rho)
    for a in range(1, 9):
        nb = np.roll(np.roll(psi, -EY[a], axis=0), -EX[a], axis=1)  # psi(x + e_a)
        Sx += W_FORCE[a] * nb * EX[a]
        Sy += W_FORCE[a] * nb * EY[a]
    return psi, -G * psi * Sx, -G * psi * Sy, -G * Sx, -G * Sy


def velocity_space_mrt_step(f, s, sigma, psi_of_rho, G):
    """Eq. 1 written in velocity space: f* = f - Lb (f - f_eq) + (S - Lb S / 2), then
    periodic streaming; Lb = M^-1 diag(s) M, S = M^-1 Sbar with Sbar from Eq. 25."""
    M = moment_basis()
    Minv = np.linalg.inv(M)
    s = np.array(s, float)
    Lb = Minv @ np.diag(s) @ M
    rho = f.sum(axis=0)
    psi, Fx, Fy, fpx, fpy = psi_F(rho, psi_of_rho, G)
    jx = np.tensordot(EX, f, axes=1)
    jy = np.tensordot(EY, f, axes=1)
    ux = (jx + 0.5 * Fx) / rho
    uy = (jy + 0.5 * Fy) / rho
    vF = ux * Fx + uy * Fy
    F2p = fpx ** 2 + fpy ** 2
    tau_e, tau_z = 1 / s[1], 1 / s[2]
    Sbar = np.array([0 * rho, 6 * vF + 12 * sigma * F2p / (tau_e - 0.5),
                     -6 * vF - 12 * sigma * F2p / (tau_z - 0.5), Fx, -Fx, Fy, -Fy,
                     2 * (ux * Fx - uy * Fy), ux * Fy + uy * Fx])
    S = np.tensordot(Minv, Sbar, axes=1)
    fe = feq(rho, ux, uy)
    fs = f - np.tensordot(Lb, f - fe, axes=1) + S - 0.5 * np.tensordot(Lb, S, axes=1)
    return stream_periodic(fs)


def bgk_guo_step(f, tau, psi_of_rho, G):
    """BGK with Guo forcing: f* = f - (f - f_eq)/tau + (1 - 1/(2 tau)) S_guo, streamed."""
    rho = f.sum(axis=0)
    psi, Fx, Fy, _, _ = psi_F(rho, psi_of_rho, G)
    jx = np.tensordot(EX, f, axes=1)
    jy = np.tensordot(EY, f, axes=1)
    ux = (jx + 0.5 * Fx) / rho
    uy = (jy + 0.5 * Fy) / rho
    fs = f - (f - feq(rho, ux, uy)) / tau + (1 - 0.5 / tau) * guo_source(ux, uy, Fx, Fy)
    return stream_periodic(fs)
