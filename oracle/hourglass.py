"""Hourglass control for 1-point H8 elements (FP64 oracle).

The paper applies "an hourglass control algorithm" to its reduced-integration
bricks and cites its source without giving formulas (Sec. 5.1).  Reading used
here (and by the CUDA library): displacement-based, Flanagan-Belytschko-type
control in total Lagrangian form.

* base vectors over the 8 nodes (natural coordinates xi_a of each node):
    h1 = xi eta,  h2 = eta zeta,  h3 = zeta xi,  h4 = xi eta zeta
* gamma_alpha = h_alpha - sum_j (h_alpha . X_{:,j}) 0B_{j,:}
  with X the reference node coordinates and 0B = 0J^-1 H_xi (Eq. 6); gamma is
  orthogonal to constant and linear nodal fields.
* stiffness k = kappa_hg (lambda + 2 mu) 0V sum_{j,a} 0B_{ja}^2 / 8,
  lambda + 2 mu = kappa + 4 mu / 3.
* energy  W_hg = k / 2 sum_alpha sum_i (gamma_alpha . u_{:,i})^2
  force   f_hg[a, i] = dW_hg / du_{a,i} = k sum_alpha gamma_{alpha,a} (gamma_alpha . u_{:,i}).

The force is zero for rigid motions and every linear displacement field, so it
leaves the patch test of the 1-point element intact.
"""
import numpy as np

from . import elements

_xi = elements.XI_HEX8
H_ALPHA = np.stack([_xi[:, 0] * _xi[:, 1], _xi[:, 1] * _xi[:, 2],
                    _xi[:, 2] * _xi[:, 0], _xi[:, 0] * _xi[:, 1] * _xi[:, 2]])  # (4, 8)


def hourglass_constants(X, conn, mu, kappa, hg_coeff):
    """gamma (E, 4, 8) and k (E,) for every H8 element."""
    J0 = elements.reference_jacobian(X, conn, elements.HEX8)
    B0 = np.linalg.solve(J0, np.broadcast_to(elements.HXI_HEX8, (J0.shape[0], 3, 8)))
    V0 = elements.element_volume(np.linalg.det(J0), elements.HEX8)
    Xe = X[conn]                                                    # (E, 8, 3)
    hx = np.einsum("qa,eaj->eqj", H_ALPHA, Xe)                      # h_alpha . X_{:,j}
    gamma = H_ALPHA[None] - np.einsum("eqj,eja->eqa", hx, B0)
    lam2mu = np.asarray(kappa) + 4.0 / 3.0 * np.asarray(mu)
    k = hg_coeff * lam2mu * V0 * np.einsum("eja,eja->e", B0, B0) / 8.0
    return gamma, k


def hourglass_forces(u_e, gamma, k):
    """f_hg (E, 8, 3) for element displacements u_e (E, 8, 3)."""
    q = np.einsum("eqb,ebi->eqi", gamma, u_e)                       # gamma_alpha . u_{:,i}
    return k[:, None, None] * np.einsum("eqa,eqi->eai", gamma, q)


def hourglass_energy(u_e, gamma, k):
    q = np.einsum("eqb,ebi->eqi", gamma, u_e)
    return 0.5 * k * np.einsum("eqi,eqi->e", q, q)
