"""A second, independent restatement of one time step, for brute-force checks
of the oracle on tiny grids (test code only).

It is written differently from the oracle on purpose:
- the moment matrix is built from the polynomial definitions of the moments
  (Lallemand and Luo, ref. [25]) evaluated on the velocity set of Eq. 8, and
  inverted with numpy.linalg.inv;
- equilibria are taken in velocity space (Eq. 13 and Eq. 37 first occurrence)
  and projected, m_eq = M f_eq; the forcing is the Guo-Zhao velocity-space
  term projected, S = M S~ (the form the paper's Section 3.1 reviews);
- streaming uses np.roll over whole planes;
- the wall rule is vectorised over each edge.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0


def velocities():
    ex = [0.0]
    ey = [0.0]
    for i in range(1, 5):
        ex.append(np.cos((i - 1) * np.pi / 2))
        ey.append(np.sin((i - 1) * np.pi / 2))
    for i in range(5, 9):
        ex.append(np.sqrt(2) * np.cos((2 * i - 9) * np.pi / 4))
        ey.append(np.sqrt(2) * np.sin((2 * i - 9) * np.pi / 4))
    return np.rint(ex).astype(int), np.rint(ey).astype(int)


EX, EY = velocities()
EX5, EY5 = EX[:5], EY[:5]
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def moment_matrix():
    e2 = EX ** 2 + EY ** 2
    rows = [np.ones(9), -4 + 3 * e2, 4 - 10.5 * e2 + 4.5 * e2 ** 2, EX, (-5 + 3 * e2) * EX,
            EY, (-5 + 3 * e2) * EY, EX ** 2 - EY ** 2, EX * EY]
    return np.array(rows, dtype=float)


def thermal_matrix():
    e2 = EX5 ** 2 + EY5 ** 2
    return np.array([np.ones(5), EX5, EY5, -4 + 5 * e2, EX5 ** 2 - EY5 ** 2], dtype=float)


M = moment_matrix()
MI = np.linalg.inv(M)
N = thermal_matrix()
NI = np.linalg.inv(N)


def _col(v, like):
    """Reshapes a per-direction vector to broadcast against a field of shape like."""
    return np.asarray(v).reshape((-1,) + (1,) * np.ndim(like))


def feq(rho0, P, ux, uy, phi):
    """Eq. 13-14 over whole fields; returns (9, ...)."""
    ux, uy = np.asarray(ux, float), np.asarray(uy, float)
    eu = _col(EX, ux) * ux + _col(EY, ux) * uy
    uu = ux * ux + uy * uy
    Wc = _col(W, ux)
    s = Wc * (eu / CS2 + eu * eu / (2 * phi * CS2 ** 2) - uu / (2 * phi * CS2))
    out = Wc * P / CS2 + rho0 * s
    out[0] = rho0 - (1 - W[0]) * P / CS2 + rho0 * s[0]
    return out


def geq(T, ux, uy, sigma, varpi):
    ux, uy = np.asarray(ux, float), np.asarray(uy, float)
    w5 = np.array([(1 - varpi) / 5] + [(4 + varpi) / 20] * 4)
    c2 = (4 + varpi) / 10
    eu = _col(EX5, ux) * ux + _col(EY5, ux) * uy
    return _col(w5, ux) * T * (1 + eu / (sigma * c2))


def guo_source(rho0, ux, uy, Fx, Fy, phi):
    ux, uy = np.asarray(ux, float), np.asarray(uy, float)
    eu = _col(EX, ux) * ux + _col(EY, ux) * uy
    eF = _col(EX, ux) * Fx + _col(EY, ux) * Fy
    uF = ux * Fx + uy * Fy
    return _col(W, ux) * rho0 * (eF / CS2 + eu * eF / (phi * CS2 ** 2) - uF / (phi * CS2))


def ergun_field(phi, phi_bar, K_bar, forchheimer=True):
    """Per-cell K and F_phi of Eq. 5 for a porosity field, with the particle
    diameter fixed by K(phi_bar) = K_bar."""
    phi = np.asarray(phi, float)
    if phi.ndim == 0 and phi == phi_bar:  # uniform porosity: K_bar itself (also at phi = 1)
        K = np.float64(K_bar)
    else:
        K = K_bar * (phi / phi_bar) ** 3 * ((1 - phi_bar) / (1 - phi)) ** 2
    Fphi = 1.75 / np.sqrt(150 * phi ** 3) if forchheimer else np.zeros_like(phi)
    return K, Fphi


class Restated:
    """Cavity with walls on all four edges.  p["phi"], p["K"], p["Fphi"] are
    scalars or (ny, nx) fields; p.get("thermal_bc"): 0 side-heated (T_h left,
    T_c right, adiabatic top and bottom), 1 every wall at T_c;
    p.get("adiabatic_order"): 1 (T_b = T_f) or 2 (T_b = (4 T_f - T_ff) / 3)."""

    def __init__(self, p: dict):
        self.p = p

    def _macros(self, f, g):
        p = self.p
        T = g.sum(0) + 0.5 * p["Q"] / p["sigma"]
        Gy = p["gbeta"] * (T - p["T0"]) + p["Gy"]
        Gx = np.full_like(T, p["Gx"])
        phi, K, nu, Fphi = p["phi"], p["K"], p["nu"], p["Fphi"]
        vx = np.tensordot(EX, f, axes=1) / p["rho0"] + 0.5 * phi * Gx
        vy = np.tensordot(EY, f, axes=1) / p["rho0"] + 0.5 * phi * Gy
        l0 = 0.5 * (1 + phi * 0.5 * nu / K)
        l1 = phi * 0.5 * Fphi / np.sqrt(K)
        den = l0 + np.sqrt(l0 * l0 + l1 * np.hypot(vx, vy))
        ux, uy = vx / den, vy / den
        uu = ux * ux + uy * uy
        s0 = W[0] * (-uu / (2 * phi * CS2))
        P = CS2 / (1 - W[0]) * (f[1:].sum(0) + p["rho0"] * s0)  # phi * p, Eq. 23
        return ux, uy, P, T, Gx, Gy

    def _edges(self, ny, nx):
        """(wall mask, inward dx, inward dy)."""
        dx = np.zeros((ny, nx), int)
        dy = np.zeros((ny, nx), int)
        dx[:, 0], dx[:, -1] = 1, -1
        dy[0, :], dy[-1, :] = 1, -1
        return (dx != 0) | (dy != 0), dx, dy

    def imposed(self, f, g):
        """(P_b, T_b) on every node (meaningful on walls) from the inner neighbours."""
        p = self.p
        ny, nx = f.shape[1:]
        wall, dx, dy = self._edges(ny, nx)
        ux, uy, P, T, _, _ = self._macros(f, g)
        yy, xx = np.indices((ny, nx))
        yf, xf = yy + dy, xx + dx
        phi = np.broadcast_to(np.asarray(p["phi"], float), (ny, nx))
        Pb = phi * P[yf, xf] / phi[yf, xf]  # p_b = p_f with P = phi p
        if p.get("adiabatic_order", 1) == 2:
            yff, xff = np.clip(yy + 2 * dy, 0, ny - 1), np.clip(xx + 2 * dx, 0, nx - 1)
            Tb = (4 * T[yf, xf] - T[yff, xff]) / 3
        else:
            Tb = T[yf, xf].copy()
        if p.get("thermal_bc", 0) == 1:
            Tb[:] = p["Tc"]
        else:
            Tb[:, 0] = p["Th"]
            Tb[:, -1] = p["Tc"]
        return Pb, Tb

    def wall_rule(self, f, g):
        p = self.p
        ny, nx = f.shape[1:]
        wall, dx, dy = self._edges(ny, nx)
        ux, uy, P, T, _, _ = self._macros(f, g)
        fneq = f - feq(p["rho0"], P, ux, uy, p["phi"])
        gneq = g - geq(T, ux, uy, p["sigma"], p["varpi"])
        Pb, Tb = self.imposed(f, g)
        yy, xx = np.indices((ny, nx))
        yf, xf = yy + dy, xx + dx
        z = np.zeros((ny, nx))
        fb = feq(p["rho0"], Pb, z, z, p["phi"]) + fneq[:, yf, xf]
        gb = geq(Tb, z, z, p["sigma"], p["varpi"]) + gneq[:, yf, xf]
        f = np.where(wall[None], fb, f)
        g = np.where(wall[None], gb, g)
        return f, g, Pb, Tb

    def step(self, f, g, Pb, Tb):
        p = self.p
        ny, nx = f.shape[1:]
        wall, _, _ = self._edges(ny, nx)
        ux, uy, P, T, Gx, Gy = self._macros(f, g)
        ux = np.where(wall, 0.0, ux)
        uy = np.where(wall, 0.0, uy)
        P = np.where(wall, Pb, P)
        T = np.where(wall, Tb, T)
        Gy = p["gbeta"] * (T - p["T0"]) + p["Gy"]
        phi, K, nu, Fphi = p["phi"], p["K"], p["nu"], p["Fphi"]
        um = np.hypot(ux, uy)
        Fx = -phi * nu / K * ux - phi * Fphi / np.sqrt(K) * um * ux + phi * Gx
        Fy = -phi * nu / K * uy - phi * Fphi / np.sqrt(K) * um * uy + phi * Gy
        s = np.asarray(p["s"])[:, None, None]
        z = np.asarray(p["zeta"])[:, None, None]
        m = np.tensordot(M, f, axes=1)
        meq = np.tensordot(M, feq(p["rho0"], P, ux, uy, phi), axes=1)
        S = np.tensordot(M, guo_source(p["rho0"], ux, uy, Fx, Fy, phi), axes=1)
        fp = np.tensordot(MI, m - s * (m - meq) + (1 - s / 2) * S, axes=1)
        n = np.tensordot(N, g, axes=1)
        neq = np.tensordot(N, geq(T, ux, uy, p["sigma"], p["varpi"]), axes=1)
        psi = np.zeros_like(n)
        psi[0] = p["Q"] / p["sigma"]
        psi[3] = p["varpi"] * p["Q"] / p["sigma"]
        gp = np.tensordot(NI, n - z * (n - neq) + (1 - z / 2) * psi, axes=1)
        fs = np.stack([np.roll(np.roll(fp[i], EY[i], axis=0), EX[i], axis=1) for i in range(9)])
        gs = np.stack([np.roll(np.roll(gp[i], EY5[i], axis=0), EX5[i], axis=1) for i in range(5)])
        return self.wall_rule(fs, gs)
