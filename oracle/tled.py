"""Classical TLED nodal forces in FP64 (oracle O-B), coded independently of djtled.

Total Lagrangian element forces through the deformation gradient, the right
Cauchy-Green tensor and the second Piola-Kirchhoff stress (Eq. 1, 4, 7-8;
Sec. 7 "Comparison with TLED", Eq. 54-55 and the TLED column of Table 8):

  0B = 0J^-1 H_xi                         (Eq. 6)
  X  = I + u^T 0B^T   (X_ij = delta_ij + sum_a u_{a,i} 0B_{j,a})   (Table 8)
  C  = X^T X,  J = det X
  S  = 2 dPsi/dC                          (Eq. 7)
  F  = X S 0B 0V                          (Eq. 4)

S is built from the textbook derivatives of the modified invariants
(I1b = J^-2/3 tr C, I2b = J^-4/3 I2, I4b = J^-2/3 a.Ca, I6b = J^-2/3 b.Cb):

  dI1b/dC = J^-2/3 (I - I1/3 C^-1)
  dI2b/dC = J^-4/3 (I1 I - C - 2/3 I2 C^-1)
  dI4b/dC = J^-2/3 (A - I4/3 C^-1)
  dJ/dC   = J/2 C^-1

so this module never touches the G matrices, m-vectors or I_im tensors.
"""
import numpy as np

from . import elements

NH, TI, OT, MR = 0, 1, 2, 3


def _unit_outer(d):
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d, axis=-1, keepdims=True)
    return d, np.einsum("ei,ej->eij", d, d)


def shape_derivatives(X, conn, elem_type):
    """0B = 0J^-1 H_xi (Eq. 6) and 0V."""
    J0 = elements.reference_jacobian(X, conn, elem_type)
    B0 = np.linalg.solve(J0, np.broadcast_to(elements.Hxi(elem_type), (J0.shape[0],) +
                                              elements.Hxi(elem_type).shape))
    V0 = elements.element_volume(np.linalg.det(J0), elem_type)
    return B0, V0


def deformation(u_e, B0):
    """X = I + sum_a u_a (x) 0B[:, a] (Table 8), C, C^-1 and J = det X."""
    Xd = np.eye(3)[None] + np.einsum("eai,eja->eij", u_e, B0)
    C = np.transpose(Xd, (0, 2, 1)) @ Xd
    return Xd, C, np.linalg.inv(C), np.linalg.det(Xd)


def second_pk_stress(C, Cinv, J, mat, a_dir, b_dir):
    """S = 2 dPsi/dC for the models of Table 3 (textbook chain rule)."""
    model = np.asarray(mat["model"])
    I = np.eye(3)[None]
    I1 = np.einsum("eii->e", C)
    I2 = 0.5 * (I1 ** 2 - np.einsum("eij,eji->e", C, C))
    _, A = _unit_outer(a_dir)
    _, B = _unit_outer(b_dir)
    I4 = np.einsum("eij,eij->e", A, C)
    I6 = np.einsum("eij,eij->e", B, C)
    Jm23 = J ** (-2.0 / 3.0)
    Jm43 = J ** (-4.0 / 3.0)
    c = lambda s: s[:, None, None]
    dI1 = c(Jm23) * (I - c(I1 / 3.0) * Cinv)
    dI2 = c(Jm43) * (c(I1) * I - C - c(2.0 / 3.0 * I2) * Cinv)
    dI4 = c(Jm23) * (A - c(I4 / 3.0) * Cinv)
    dI6 = c(Jm23) * (B - c(I6 / 3.0) * Cinv)
    dJ = c(0.5 * J) * Cinv
    psi1 = 0.5 * mat["mu"]
    psi2 = np.where(model == MR, mat["c01"], 0.0)
    psi4 = np.where((model == TI) | (model == OT), mat["eta_a"] * (Jm23 * I4 - 1.0), 0.0)
    psi6 = np.where(model == OT, mat["eta_b"] * (Jm23 * I6 - 1.0), 0.0)
    psiJ = mat["kappa"] * (J - 1.0)
    return 2.0 * (c(psi1) * dI1 + c(psi2) * dI2 + c(psi4) * dI4 + c(psi6) * dI6 + c(psiJ) * dJ)


def element_forces(u_e, X, conn, elem_type, mat, a_dir, b_dir):
    """F = X S 0B 0V (Eq. 4); returned as (E, n_e, 3), row a = force on node a."""
    B0, V0 = shape_derivatives(X, conn, elem_type)
    Xd, C, Cinv, J = deformation(u_e, B0)
    S = second_pk_stress(C, Cinv, J, mat, a_dir, b_dir)
    F = Xd @ S @ B0 * V0[:, None, None]
    return np.transpose(F, (0, 2, 1))


def strain_energy(u_e, X, conn, elem_type, mat, a_dir, b_dir):
    """0V Psi per element (Table 3 energies), from C directly."""
    B0, V0 = shape_derivatives(X, conn, elem_type)
    Xd, C, Cinv, J = deformation(u_e, B0)
    model = np.asarray(mat["model"])
    I1 = np.einsum("eii->e", C)
    I2 = 0.5 * (I1 ** 2 - np.einsum("eij,eji->e", C, C))
    _, A = _unit_outer(a_dir)
    _, B = _unit_outer(b_dir)
    I4 = np.einsum("eij,eij->e", A, C)
    I6 = np.einsum("eij,eij->e", B, C)
    Jm23 = J ** (-2.0 / 3.0)
    psi = 0.5 * mat["mu"] * (Jm23 * I1 - 3.0) + 0.5 * mat["kappa"] * (J - 1.0) ** 2
    psi = psi + np.where(model == MR, mat["c01"] * (J ** (-4.0 / 3.0) * I2 - 3.0), 0.0)
    psi = psi + np.where((model == TI) | (model == OT),
                         0.5 * mat["eta_a"] * (Jm23 * I4 - 1.0) ** 2, 0.0)
    psi = psi + np.where(model == OT, 0.5 * mat["eta_b"] * (Jm23 * I6 - 1.0) ** 2, 0.0)
    return V0 * psi
