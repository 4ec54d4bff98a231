"""Element geometry for the oracle: H_xi, 0J and 0V (FP64).

* T4 uses volume coordinates of the unit tetrahedron in natural space
  (Sec. 7, last paragraph): N = [1 - xi - eta - zeta, xi, eta, zeta].
* H8 uses trilinear N_a = (1 + xi_a xi)(1 + eta_a eta)(1 + zeta_a zeta) / 8 with
  natural coordinates in [-1, 1] (Sec. 2.1.2) and 1-point Gauss integration at
  the centre (Sec. 1 and Sec. 5.1), so H_xi[i, a] = xi_{a,i} / 8.
"""
import numpy as np

TET4 = 4
HEX8 = 8

# rows: d/dxi, d/deta, d/dzeta ; columns: local node a
HXI_TET4 = np.array([[-1.0, 1.0, 0.0, 0.0],
                     [-1.0, 0.0, 1.0, 0.0],
                     [-1.0, 0.0, 0.0, 1.0]])

# natural coordinates of the 8 brick nodes: bottom face counter-clockwise, then top
XI_HEX8 = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                    [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)
HXI_HEX8 = XI_HEX8.T / 8.0


def Hxi(elem_type: int) -> np.ndarray:
    """Natural derivatives of the interpolation functions, shape (3, n_e) (Eq. 6)."""
    if elem_type == TET4:
        return HXI_TET4
    if elem_type == HEX8:
        return HXI_HEX8
    raise ValueError(f"unknown element type {elem_type}")


def element_nodes(X: np.ndarray, conn: np.ndarray) -> np.ndarray:
    """Reference node coordinates per element, shape (E, n_e, 3)."""
    return X[conn]


def reference_jacobian(X: np.ndarray, conn: np.ndarray, elem_type: int) -> np.ndarray:
    """0J[i, j] = d x_j / d xi_i = sum_a H_xi[i, a] x_{a, j}  (Eq. 3), shape (E, 3, 3)."""
    return np.einsum("ia,eaj->eij", Hxi(elem_type), element_nodes(X, conn))


def element_volume(detJ0: np.ndarray, elem_type: int) -> np.ndarray:
    """Initial element volume 0V.

    T4: the unit tetrahedron has volume 1/6, so 0V = det(0J) / 6.
    H8: 1-point Gauss rule of weight 8 on [-1, 1]^3, so 0V = 8 det(0J) (exact
    for parallelepipeds).
    """
    if elem_type == TET4:
        return detJ0 / 6.0
    return 8.0 * detJ0
