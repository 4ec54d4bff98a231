"""Paper-literal DJ-TLED nodal forces in FP64 (oracle O-A).

Follows Algorithm 1 of the paper in its order:

pre-computation (per element)
  1. 0J, det(0J), 0V, A, B and H_xi                       (Eq. 3, 6, 30)
  2. the six G matrices                                    (App. B, Eq. B.1-B.6)
  3. m1, m4, m6 and M2 (W)                                 (App. C, Eq. C.1-C.5)
  4. I1m, I2m, I4m, I6m                                    (Table 2, Eq. 37, 41, 45, 46)
run time (per element)
  1. tJ (Eq. 11), tJ^-1 and J (Eq. 12)
  2. g_hat (Eq. 17-18)
  3. I1, I2, I4, I6 (Table 1) and the modified invariants (Table 1, note 1)
  4. the nodal force contributions (Table 3)

Reading of Eq. 11: with 0J oriented as in Eq. 3 (row i = d/d xi_i, column
j = coordinate j), the update is tJ = 0J + H_xi u_e where u_e is the (n_e, 3)
matrix of nodal displacements.  Written as "u H_xi^T" with u of shape (3, n_e),
Eq. 11 would give the transpose; Eq. 5, 6, 9 and A.6 are only consistent with
the Eq. 3 orientation, and the TLED pin (tests) confirms it.

The I5/I7 terms (Eq. 47-51) are not built: no model of Table 3 uses them.
"""
import numpy as np

from . import elements

# Unit symmetric patterns multiplying g11, g22, g33, g12, g13, g23 in Eq. 16.
E_KL = np.zeros((6, 3, 3))
for _k, (_i, _j) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
    E_KL[_k, _i, _j] = 1.0
    E_KL[_k, _j, _i] = 1.0

NH, TI, OT, MR = 0, 1, 2, 3


class InvertedElement(ValueError):
    pass


def structural_matrix(d: np.ndarray) -> np.ndarray:
    """A = a a^T for unit fibre direction a (Sec. 2.3.2); input normalised here."""
    d = d / np.linalg.norm(d, axis=-1, keepdims=True)
    return np.einsum("ei,ej->eij", d, d)


def precompute(X, conn, elem_type, a_dir=None, b_dir=None, with_mr=False):
    """Pre-computation of Algorithm 1 for every element (FP64)."""
    Hxi = elements.Hxi(elem_type)
    J0 = elements.reference_jacobian(X, conn, elem_type)          # Eq. 3
    detJ0 = np.linalg.det(J0)
    if np.any(detJ0 <= 0.0):
        bad = int(np.nonzero(detJ0 <= 0.0)[0][0])
        raise InvertedElement(f"element {bad} has det(0J) <= 0")
    V0 = elements.element_volume(detJ0, elem_type)
    J0inv = np.linalg.inv(J0)
    J0invT = np.transpose(J0inv, (0, 2, 1))
    E = J0.shape[0]
    if a_dir is None:
        a_dir = np.tile([1.0, 0.0, 0.0], (E, 1))
    if b_dir is None:
        b_dir = np.tile([0.0, 1.0, 0.0], (E, 1))
    A = structural_matrix(np.asarray(a_dir, dtype=np.float64))
    B = structural_matrix(np.asarray(b_dir, dtype=np.float64))
    # App. B: G_kl = 0J^-1 E_kl 0J^-T
    G = np.einsum("eij,kjl,eml->ekim", J0inv, E_KL, J0inv)
    # App. C
    m1 = np.einsum("ekii->ek", G)                                   # C.1
    m4 = np.einsum("eij,ekji->ek", A, G)                            # C.2  tr(A G)
    m6 = np.einsum("eij,ekji->ek", B, G)                            # C.3  tr(B G)
    # Table 2
    I1m = 2.0 * V0[:, None, None] * J0invT @ J0inv                  # Eq. 37
    I4m = 2.0 * V0[:, None, None] * J0invT @ A @ J0inv              # Eq. 45
    I6m = 2.0 * V0[:, None, None] * J0invT @ B @ J0inv              # Eq. 46
    pre = dict(elem_type=elem_type, Hxi=Hxi, conn=conn, J0=J0, detJ0=detJ0, V0=V0,
               J0inv=J0inv, A=A, B=B, G=G, m1=m1, m4=m4, m6=m6,
               I1m=I1m, I4m=I4m, I6m=I6m)
    if with_mr:
        W = np.einsum("ekji,elji->ekl", G, G)                        # C.4 tr(G_k^T G_l)
        M2 = 0.5 * (np.einsum("ek,el->ekl", m1, m1) - W)            # C.5
        eye = np.eye(3)
        inner = m1[:, :, None, None] * eye[None, None] - G          # tr(G_k) I - G_k
        I2m = 2.0 * V0[:, None, None, None] * np.einsum(
            "eji,ekjl,elm->ekim", J0inv, inner, J0inv)              # Eq. 41a-f
        pre.update(W=W, M2=M2, I2m=I2m)
    return pre


def g_hat(tJ: np.ndarray) -> np.ndarray:
    """g_hat = [g11 g22 g33 g12 g13 g23] of tJ tJ^T  (Eq. 17-18)."""
    g = tJ @ np.transpose(tJ, (0, 2, 1))
    return np.stack([g[:, 0, 0], g[:, 1, 1], g[:, 2, 2],
                     g[:, 0, 1], g[:, 0, 2], g[:, 1, 2]], axis=1)


def kinematics(u_e: np.ndarray, pre: dict):
    """Runtime step 1-3: tJ, tJ^-1, J, g_hat and the invariants."""
    tJ = pre["J0"] + np.einsum("ia,eaj->eij", pre["Hxi"], u_e)      # Eq. 11 (Eq. 3 orientation)
    detJ = np.linalg.det(tJ)
    J = detJ / pre["detJ0"]                                          # Eq. 12
    gh = g_hat(tJ)                                                   # Eq. 18
    I1 = np.einsum("ek,ek->e", gh, pre["m1"])                        # Eq. 27
    I4 = np.einsum("ek,ek->e", gh, pre["m4"])                        # Eq. 31
    I6 = np.einsum("ek,ek->e", gh, pre["m6"])                        # Eq. 32
    out = dict(tJ=tJ, detJ=detJ, J=J, g_hat=gh, I1=I1, I4=I4, I6=I6)
    if "M2" in pre:
        out["I2"] = np.einsum("ek,ekl,el->e", gh, pre["M2"], gh)    # Eq. 28
    return out


def element_forces(u_e: np.ndarray, pre: dict, mat: dict, pressure=None) -> np.ndarray:
    """Nodal force contributions of every element (Table 3), shape (E, n_e, 3).

    mat: model (E,), mu, kappa, eta_a, eta_b, c01 (E,).  For MR, C10 = mu / 2.
    Generic form (Table 3, rows "Psi(I1, I2, I4, I6) + Psi(J)"):

      F = ( J^-2/3 tJ^T ( dPsi/dI1 I1m + dPsi/dI4 I4m + dPsi/dI6 I6m
                          + J^-2/3 dPsi/dI2 (g_hat^T . I2m) )
            + ( -2/3 ( dPsi/dI1 I1 + dPsi/dI4 I4 + dPsi/dI6 I6 + 2 dPsi/dI2 I2 )
                + J dPsi/dJ ) 0V tJ^-1 ) H_xi

    with Psi = mu/2 (I1-3) + C01 (I2-3) + eta_a/2 (I4-1)^2 + eta_b/2 (I6-1)^2
    + kappa/2 (J-1)^2 (all invariants modified), which gives the NH, TI, OT and
    MR rows of Table 3.  Row a of the result is the force on local node a.

    pressure (E,), optional: replaces dPsi/dJ = kappa (J - 1) (average nodal
    pressure, oracle/anp.py).
    """
    k = kinematics(u_e, pre)
    J = k["J"]
    if np.any(k["detJ"] <= 0.0):
        bad = int(np.nonzero(k["detJ"] <= 0.0)[0][0])
        raise InvertedElement(f"element {bad} inverted (det tJ <= 0)")
    Jm23 = J ** (-2.0 / 3.0)
    model = np.asarray(mat["model"])
    I1b = Jm23 * k["I1"]                                             # Table 1 note
    I4b = Jm23 * k["I4"]
    I6b = Jm23 * k["I6"]
    dPsi1 = 0.5 * mat["mu"]
    dPsi4 = np.where((model == TI) | (model == OT), mat["eta_a"] * (I4b - 1.0), 0.0)
    dPsi6 = np.where(model == OT, mat["eta_b"] * (I6b - 1.0), 0.0)
    JdPsiJ = mat["kappa"] * J * (J - 1.0) if pressure is None else J * np.asarray(pressure)
    dev = (dPsi1[:, None, None] * pre["I1m"] + dPsi4[:, None, None] * pre["I4m"]
           + dPsi6[:, None, None] * pre["I6m"])
    vol_coef = -2.0 / 3.0 * (dPsi1 * I1b + dPsi4 * I4b + dPsi6 * I6b) + JdPsiJ
    if np.any(model == MR):
        if "I2m" not in pre:
            raise ValueError("MR elements need precompute(..., with_mr=True)")
        I2b = J ** (-4.0 / 3.0) * k["I2"]                            # Table 1 note
        dPsi2 = np.where(model == MR, mat["c01"], 0.0)
        gI2m = np.einsum("ek,ekij->eij", k["g_hat"], pre["I2m"])     # Eq. 42
        dev = dev + (Jm23 * dPsi2)[:, None, None] * gI2m
        vol_coef = vol_coef - 2.0 / 3.0 * 2.0 * dPsi2 * I2b
    tJT = np.transpose(k["tJ"], (0, 2, 1))
    tJinv = np.linalg.inv(k["tJ"])
    Fmat = Jm23[:, None, None] * (tJT @ dev) \
        + (vol_coef * pre["V0"])[:, None, None] * tJinv
    F = Fmat @ pre["Hxi"]                                            # (E, 3, n_e)
    return np.transpose(F, (0, 2, 1))


def strain_energy_density(k: dict, mat: dict, with_mr: bool = False) -> np.ndarray:
    """Psi per element from the invariants of Table 1 (models of Table 3)."""
    J = k["J"]
    model = np.asarray(mat["model"])
    Jm23 = J ** (-2.0 / 3.0)
    psi = 0.5 * mat["mu"] * (Jm23 * k["I1"] - 3.0) + 0.5 * mat["kappa"] * (J - 1.0) ** 2
    fa = (model == TI) | (model == OT)
    psi = psi + np.where(fa, 0.5 * mat["eta_a"] * (Jm23 * k["I4"] - 1.0) ** 2, 0.0)
    psi = psi + np.where(model == OT, 0.5 * mat["eta_b"] * (Jm23 * k["I6"] - 1.0) ** 2, 0.0)
    if with_mr:
        psi = psi + np.where(model == MR, mat["c01"] * (J ** (-4.0 / 3.0) * k["I2"] - 3.0), 0.0)
    return psi
