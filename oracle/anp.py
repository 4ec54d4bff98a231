"""Average nodal pressure (ANP) for linear tetrahedra, FP64 (oracle, test
infrastructure only: imported by tests/, smoke() and the benchmark's CPU
baseline, never by the CUDA library's path).

Sec. 7 names ANP as the remedy for volumetric locking of nearly
incompressible T4 meshes and leaves it unbuilt ("could be constructed from the
TLED implementation").  Reading used here, the average-nodal-pressure
tetrahedron that the cited work applies to TLED, written in this project's
notation (volumetric energy kappa/2 (J - 1)^2 per unit reference volume, as
in Table 3):

  reference nodal volume   V0_i = sum_{e at i} 0V_e / 4
  current nodal volume     V_i  = sum_{e at i} J_e 0V_e / 4
  nodal volume ratio       J_i  = V_i / V0_i
  nodal bulk modulus       kappa_i = sum_{e at i} kappa_e 0V_e / 4 / V0_i
  nodal pressure           p_i  = kappa_i (J_i - 1)
  element pressure         pbar_e = (1/4) sum_{i in e} p_i

and in the element force (Table 3) the volumetric factor kappa (J - 1) is
replaced by pbar_e; the isochoric part is unchanged.  These forces are the
gradient of  sum_e 0V_e Psi_iso,e + sum_i kappa_i V0_i / 2 (J_i - 1)^2.
"""
import numpy as np


def nodal_constants(V0, kappa, conn, n_nodes):
    """V0_i and kappa_i of every node (element volumes and bulk moduli)."""
    conn = np.asarray(conn)
    ne = conn.shape[1]
    V0n = np.zeros(n_nodes)
    np.add.at(V0n, conn.ravel(), np.repeat(np.asarray(V0) / ne, ne))
    kV0n = np.zeros(n_nodes)
    np.add.at(kV0n, conn.ravel(), np.repeat(np.asarray(kappa) * np.asarray(V0) / ne, ne))
    with np.errstate(invalid="ignore", divide="ignore"):
        kn = np.where(V0n > 0, kV0n / V0n, 0.0)
    return V0n, kn


def nodal_pressure(J, V0, kappa, conn, n_nodes):
    """p_i = kappa_i (J_i - 1) with J_i the ratio of current to reference nodal
    volume (element volumes J_e 0V_e shared equally by the element's nodes)."""
    conn = np.asarray(conn)
    ne = conn.shape[1]
    V0n, kn = nodal_constants(V0, kappa, conn, n_nodes)
    Vn = np.zeros(n_nodes)
    np.add.at(Vn, conn.ravel(), np.repeat(np.asarray(J) * np.asarray(V0) / ne, ne))
    with np.errstate(invalid="ignore", divide="ignore"):
        Jn = np.where(V0n > 0, Vn / V0n, 1.0)
    return kn * (Jn - 1.0)


def element_pressure(J, V0, kappa, conn, n_nodes):
    """pbar_e: mean of the nodal pressures over the element's nodes."""
    p = nodal_pressure(J, V0, kappa, conn, n_nodes)
    return p[np.asarray(conn)].mean(axis=1)


def volumetric_energy(J, V0, kappa, conn, n_nodes):
    """sum_i kappa_i V0_i / 2 (J_i - 1)^2 (the energy whose gradient the ANP
    volumetric forces are)."""
    conn = np.asarray(conn)
    ne = conn.shape[1]
    V0n, kn = nodal_constants(V0, kappa, conn, n_nodes)
    Vn = np.zeros(n_nodes)
    np.add.at(Vn, conn.ravel(), np.repeat(np.asarray(J) * np.asarray(V0) / ne, ne))
    used = V0n > 0
    Jn = Vn[used] / V0n[used]
    return float(np.sum(0.5 * kn[used] * V0n[used] * (Jn - 1.0) ** 2))
