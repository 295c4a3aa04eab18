"""Small analytic initial states used by the oracle pins and parity tests."""
import numpy as np

from paper_1110_0740_gb300 import workloads as W

G53 = 5.0 / 3.0


def primitive_jacobian_7(V, gamma):
    """The 7x7 primitive Jacobian of the 1-D ideal MHD system (Eq. 1 of the
    paper) on (rho, v_n, v_t1, v_t2, p, B_t1, B_t2), B_n a parameter, written
    from the PDE: rho_t + u rho_x + rho u_x = 0, rho(v_t + u v_x) + grad p_t
    - B_n B_x = 0, p_t + u p_x + gamma p u_x = 0, B_t = curl(v x B)."""
    rho, u, p, Bn, B1, B2 = V[0], V[1], V[4], V[5], V[6], V[7]
    return np.array([
        [u, rho, 0, 0, 0, 0, 0],
        [0, u, 0, 0, 1 / rho, B1 / rho, B2 / rho],
        [0, 0, u, 0, 0, -Bn / rho, 0],
        [0, 0, 0, u, 0, 0, -Bn / rho],
        [0, gamma * p, 0, 0, u, 0, 0],
        [0, B1, -Bn, 0, 0, u, 0],
        [0, B2, 0, -Bn, 0, 0, u],
    ], dtype=np.float64)


IDX7 = [0, 1, 2, 3, 4, 6, 7]


def oblique_wave_2d(N, wave, gamma=G53, eps=1e-6):
    """Linear eigenmode of ideal MHD travelling along (1,1)/sqrt(2) on the
    periodic unit square.  The eigenvector comes from numpy.linalg.eig of the
    primitive Jacobian above (independent of the oracle's eigenvectors).
    Returns (U_ghosted, U_exact_interior_after_one_period, period)."""
    V0 = np.array([1.0, 0.0, 0.0, 0.0, 1.0 / gamma, 1.0, np.sqrt(2.0), 0.5, 0.0])
    if wave == "entropy":
        V0[1] = 1.0
    A = primitive_jacobian_7(V0, gamma)
    lam, R = np.linalg.eig(A)
    order = np.argsort(lam.real)
    lam, R = lam.real[order], R.real[:, order]
    k = {"fast": 6, "alfven": 5, "slow": 4, "entropy": 3}[wave]
    c, r = lam[k], R[:, k]
    nh = np.array([1.0, 1.0]) / np.sqrt(2.0)
    t1 = np.array([-1.0, 1.0]) / np.sqrt(2.0)
    x = (np.arange(N) + 0.5) / N
    X, Y = np.meshgrid(x, x, indexing="xy")
    d = eps * np.cos(2.0 * np.pi * (X + Y))
    rho = V0[0] + r[0] * d
    un = V0[1] + r[1] * d
    ut1 = r[2] * d
    ut2 = r[3] * d
    p = V0[4] + r[4] * d
    Bt1 = V0[6] + r[5] * d
    Bt2 = V0[7] + r[6] * d
    vx = un * nh[0] + ut1 * t1[0]
    vy = un * nh[1] + ut1 * t1[1]
    Bx = V0[5] * nh[0] + Bt1 * t1[0]
    By = V0[5] * nh[1] + Bt1 * t1[1]
    z = np.zeros_like(rho)
    U = W.ideal_cons([rho, vx, vy, ut2, p, Bx, By, Bt2, z], gamma)[:, None]
    period = (1.0 / np.sqrt(2.0)) / abs(c)
    return W.pad_periodic(U, 2), U, period


def mirror_x(U):
    """x -> -x: reverse x, negate m_x and B_x (psi is even)."""
    M = U[..., ::-1].copy()
    M[1] *= -1.0
    M[5] *= -1.0
    return M


def mirror_z(U):
    M = U[:, ::-1].copy()
    M[3] *= -1.0
    M[7] *= -1.0
    return M


def swap_xy(U):
    """Exchange x and y: transpose the (y, x) axes and swap m_x<->m_y, B_x<->B_y."""
    S = np.swapaxes(U, 2, 3).copy()
    S[[1, 2]] = S[[2, 1]]
    S[[5, 6]] = S[[6, 5]]
    return S
