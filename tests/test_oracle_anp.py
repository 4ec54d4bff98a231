"""Pins of the oracle's average nodal pressure (oracle/anp.py, T4).

* Homogeneous deformation: every element and node has the same volume ratio,
  so ANP must reproduce the element formulation (Table 3) exactly.
* Energy: the ANP forces are the gradient of the isochoric element energies
  plus the nodal volumetric energy sum_i kappa_i V0_i / 2 (J_i - 1)^2
  (central differences, per-element bulk moduli that differ).
* Locking (Sec. 7): a slender cantilever under a tip load, against
  Euler-Bernoulli beam theory, as nu goes from 0.3 to 0.499.  The element
  formulation locks (its deflection collapses by more than an order of
  magnitude); with ANP the deflection stays within a factor 1.5 and the
  stiffness stays positive definite (no spurious zero-energy modes).
"""
import numpy as np
import pytest

from oracle import anp, djtled, dynamics
from paper_2106_14189_gb300 import workloads as W


def _problem(seed, n=700):
    p = W.random_tet_mesh_problem(n, seed=seed)
    rng = np.random.default_rng(seed + 50)
    p.kappa = p.mu * rng.uniform(10.0, 60.0, size=p.n_elems)
    return p


def test_homogeneous_deformation_reproduces_the_element_pressure():
    p = _problem(1)
    Fdef = np.array([[1.05, 0.02, -0.01], [0.03, 0.97, 0.04], [-0.02, 0.01, 1.02]])
    U = p.X @ (Fdef - np.eye(3)).T
    p.kappa = np.full(p.n_elems, float(p.kappa[0]))
    std = dynamics.Model.from_problem(p).internal_forces(U)
    p.anp = True
    m = dynamics.Model.from_problem(p)
    F = m.internal_forces(U)
    J = djtled.kinematics(U[p.conn], m.pre)["J"]
    pbar = anp.element_pressure(J, m.pre["V0"], m.mat["kappa"], p.conn, p.n_nodes)
    assert np.allclose(pbar, p.kappa * (np.linalg.det(Fdef) - 1.0), rtol=1e-12, atol=0)
    assert np.abs(F - std).max() <= 1e-12 * np.abs(std).max()


def _energy(m, U):
    u_e = U[m.conn]
    k = djtled.kinematics(u_e, m.pre)
    iso_mat = dict(m.mat)
    iso_mat["kappa"] = np.zeros_like(m.mat["kappa"])
    w_iso = float(np.sum(m.pre["V0"] * djtled.strain_energy_density(k, iso_mat)))
    return w_iso + anp.volumetric_energy(k["J"], m.pre["V0"], m.mat["kappa"], m.conn, m.N)


def test_anp_forces_are_the_energy_gradient():
    p = _problem(2, n=300)
    p.anp = True
    m = dynamics.Model.from_problem(p)
    rng = np.random.default_rng(7)
    U = rng.normal(size=(p.n_nodes, 3)) * 0.02 * np.ptp(p.X)
    F = m.internal_forces(U)
    h = 1e-6 * np.ptp(p.X)
    dofs = rng.choice(3 * p.n_nodes, size=60, replace=False)
    for d in dofs:
        Up = U.copy().reshape(-1)
        Um = Up.copy()
        Up[d] += h
        Um[d] -= h
        g = (_energy(m, Up.reshape(-1, 3)) - _energy(m, Um.reshape(-1, 3))) / (2 * h)
        assert g == pytest.approx(F.reshape(-1)[d], rel=1e-5, abs=1e-6 * np.abs(F).max())


def _cantilever(anp_on, nu):
    """Bar L x b x b (L/b = 10), Kuhn tets, end x = 0 clamped, transverse tip
    load P on the end x = L; linear response from the stiffness at U = 0
    (central differences of the internal force) and a direct solve.  Returns
    the tip deflection over beam theory and the smallest stiffness eigenvalue."""
    L, b, nx, nb = 1.0, 0.1, 20, 2
    X, conn = W.box_tet4(nx, nb, nb, L, b, b)
    E = 3000.0
    mu, kappa = W.lame_from_E_nu(E, nu)
    E_count = conn.shape[0]
    mat = dict(model=np.zeros(E_count, dtype=np.uint8), mu=np.full(E_count, mu),
               kappa=np.full(E_count, kappa), rho=np.full(E_count, 1000.0),
               eta_a=np.zeros(E_count), eta_b=np.zeros(E_count), c01=np.zeros(E_count))
    m = dynamics.Model(W.TET4, X, conn, mat, anp=anp_on)
    N = X.shape[0]
    clamped = np.flatnonzero(X[:, 0] < 1e-9)
    tip = np.flatnonzero(X[:, 0] > L - 1e-9)
    free = np.ones(3 * N, dtype=bool)
    free[np.concatenate([3 * clamped, 3 * clamped + 1, 3 * clamped + 2])] = False
    f = np.flatnonzero(free)
    h = 1e-7
    K = np.zeros((len(f), len(f)))
    for c, j in enumerate(f):
        Up = np.zeros(3 * N)
        Up[j] = h
        dF = m.internal_forces(Up.reshape(-1, 3)) - m.internal_forces(-Up.reshape(-1, 3))
        K[:, c] = dF.reshape(-1)[f] / (2 * h)
    P = 1e-3
    R = np.zeros((N, 3))
    R[tip, 2] = P / len(tip)
    u = np.zeros(3 * N)
    u[f] = np.linalg.solve(K, R.reshape(-1)[f])
    delta = float(u.reshape(-1, 3)[tip, 2].mean())
    beam = P * L ** 3 / (3.0 * E * b ** 4 / 12.0)
    return delta / beam, float(np.linalg.eigvalsh(0.5 * (K + K.T))[0])


def test_anp_relieves_volumetric_locking():
    r = {(a, nu): _cantilever(a, nu) for a in (False, True) for nu in (0.3, 0.499)}
    print({k: round(v[0], 3) for k, v in r.items()})
    for nu in (0.3, 0.499):
        assert r[(True, nu)][0] > r[(False, nu)][0]
        assert r[(True, nu)][0] < 1.0 and r[(True, nu)][1] > 0.0
    assert r[(False, 0.3)][0] > 20 * r[(False, 0.499)][0]     # the element formulation locks
    assert r[(True, 0.3)][0] < 1.5 * r[(True, 0.499)][0]      # ANP does not


def test_anp_keeps_the_critical_step():
    """Averaging lowers the volumetric stiffness: the highest eigenvalue of
    M^-1 K with ANP stays below the element formulation's, so the element
    formulation's critical step (Eq. 14) remains stable."""
    from scipy.linalg import eigh
    lam_max = {}
    for on in (False, True):
        p = W.cube_compression_tet4(n=3)
        p.anp = on
        m = dynamics.Model.from_problem(p)
        N, h = p.n_nodes, 1e-7
        K = np.zeros((3 * N, 3 * N))
        for j in range(3 * N):
            Up = np.zeros(3 * N)
            Up[j] = h
            K[:, j] = (m.internal_forces(Up.reshape(-1, 3)) - m.internal_forces(-Up.reshape(-1, 3))).reshape(-1) / (2 * h)
        lam_max[on] = eigh(0.5 * (K + K.T), np.diag(np.repeat(m.mass, 3)), eigvals_only=True)[-1]
        dt = m.critical_time_step()
    assert lam_max[True] < lam_max[False]
    assert dt < 2.0 / np.sqrt(lam_max[False])
