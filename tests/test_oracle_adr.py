"""Pins of the oracle's adaptive dynamic relaxation (oracle/dynamics.py).

The scheme's three ingredients are checked against facts that do not come
from the oracle: the Rayleigh quotient against a generalized eigensolver
(Courant-Fischer bounds, exact on eigenvectors), critical damping against
the spectral radius of the damped central-difference recurrence, the error
estimate against an exactly geometric sequence, and the whole iteration
against the exact solution and lowest eigenvalue of a linear spring chain
and against the spectrum of the linearized finite element problem.
"""
import numpy as np
import pytest
from scipy.linalg import eigh

from oracle import dynamics
from paper_2106_14189_gb300 import workloads as W


def _spd(n, rng):
    A = rng.normal(size=(n, n))
    return A @ A.T + n * np.eye(n)


def test_rayleigh_quotient_eigenvectors_and_bounds():
    rng = np.random.default_rng(3)
    N = 12                          # nodes, 3 DOFs each
    K = _spd(3 * N, rng)
    mass = rng.uniform(0.5, 2.0, size=N)
    free = np.ones(3 * N, dtype=bool)
    free[[0, 4, 17]] = False        # constrained DOFs take no part
    f = np.flatnonzero(free)
    Kf = K[np.ix_(f, f)]
    Mf = np.diag(np.repeat(mass, 3)[f])
    lam, vec = eigh(Kf, Mf)
    for j in (0, 5, len(f) - 1):
        D = np.zeros(3 * N)
        D[f] = vec[:, j]
        D[~free] = 7.0              # ignored values at constrained DOFs
        dF = np.zeros(3 * N)
        dF[f] = Kf @ vec[:, j]
        dF[~free] = -3.0
        rq = dynamics.rayleigh_quotient(D.reshape(-1, 3), dF.reshape(-1, 3), mass, free)
        assert rq == pytest.approx(lam[j], rel=1e-12)
    for _ in range(20):             # any direction: lambda_min <= RQ <= lambda_max
        D = np.zeros(3 * N)
        D[f] = rng.normal(size=len(f))
        dF = np.zeros(3 * N)
        dF[f] = Kf @ D[f]
        rq = dynamics.rayleigh_quotient(D.reshape(-1, 3), dF.reshape(-1, 3), mass, free)
        assert lam[0] * (1 - 1e-12) <= rq <= lam[-1] * (1 + 1e-12)


def _spectral_radius(omega, alpha, dt):
    """Damped central difference on m u'' + alpha m u' + m omega^2 u = 0:
    u^{n+1} = (b - a m omega^2) u^n + c u^{n-1}, written from the difference
    quotients independently of the oracle's coefficients."""
    den = 1.0 + alpha * dt / 2.0
    p = (2.0 - (omega * dt) ** 2) / den
    q = -(1.0 - alpha * dt / 2.0) / den
    return max(abs(np.roots([1.0, -p, -q])))


def test_critical_damping_minimises_the_spectral_radius():
    dt = 1.0
    for omega in (0.004, 0.01, 0.03):
        a_star = dynamics.critical_damping(omega ** 2)
        assert a_star == pytest.approx(2.0 * omega, rel=1e-15)
        grid = np.linspace(0.2, 5.0, 2401) * omega
        rho = np.array([_spectral_radius(omega, a, dt) for a in grid])
        best = grid[int(np.argmin(rho))]
        assert best == pytest.approx(a_star, rel=0.02)
        # the recurrence of the oracle's own coefficients has that radius too
        s = _DummySolver(dt)
        s.set_damping(a_star)
        M = np.array([[s.b - s.a[0] * omega ** 2, s.c], [1.0, 0.0]])
        assert max(abs(np.linalg.eigvals(M))) == pytest.approx(_spectral_radius(omega, a_star, dt),
                                                                rel=1e-9)


class _DummySolver(dynamics.ExplicitSolver):
    def __init__(self, dt):
        self.dt = dt
        self.m = type("M", (), {"mass": np.ones(1)})()


def test_error_estimate_is_exact_on_a_geometric_sequence():
    rng = np.random.default_rng(5)
    u_star = rng.normal(size=30)
    C = rng.normal(size=30)
    rho, k = 0.97, 25
    u = [u_star + C * rho ** n for n in range(0, 3 * k + 1)]
    n = 3 * k
    D_now = u[n] - u[n - k]             # change over the last interval
    D_before = u[n - k] - u[n - 2 * k]  # and over the one before
    r = dynamics.interval_ratio(np.linalg.norm(D_now), np.linalg.norm(D_before))
    assert r == pytest.approx(rho ** k, rel=1e-12)
    # |u* - u_n| = sum of all later intervals = r / (1 - r) |D_now| componentwise
    est = dynamics.error_estimate(r, np.abs(D_now).max())
    assert est == pytest.approx(np.abs(u_star - u[n]).max(), rel=1e-10)
    assert dynamics.error_estimate(1.0, 1.0) == np.inf


class _LinearChain:
    """Springs k between consecutive nodes of a chain (each axis
    independently, x, y, z with different stiffness), node 0 held."""

    def __init__(self, n, masses, kx):
        self.N = n
        self.mass = np.asarray(masses, dtype=np.float64)
        K1 = np.zeros((n, n))
        for e in range(n - 1):
            K1[e:e + 2, e:e + 2] += np.array([[1.0, -1.0], [-1.0, 1.0]])
        self.K = sum(np.kron(K1, np.diag(np.eye(3)[c])) * kx[c] for c in range(3))
        self.R = np.zeros((n, 3))
        self.R[-1] = [2.0, -1.0, 0.5]

    def internal_forces(self, U):
        return (self.K @ U.reshape(-1)).reshape(-1, 3)


def test_adaptive_relaxation_on_a_linear_chain():
    n = 24
    rng = np.random.default_rng(11)
    model = _LinearChain(n, rng.uniform(0.5, 1.5, size=n), kx=(1.0, 2.0, 0.5))
    bc_dof = np.array([0, 1, 2])
    free = np.ones(3 * n, dtype=bool)
    free[bc_dof] = False
    f = np.flatnonzero(free)
    Kf = model.K[np.ix_(f, f)]
    lam = eigh(Kf, np.diag(np.repeat(model.mass, 3)[f]), eigvals_only=True)
    dt = 0.9 * 2.0 / np.sqrt(lam[-1])
    U_exact = np.zeros(3 * n)
    U_exact[f] = np.linalg.solve(Kf, model.R.reshape(-1)[f])

    def solver(alpha):
        return dynamics.ExplicitSolver(model, bc_dof, np.zeros(3), dt=dt, alpha=alpha)

    s = solver(0.0)
    steps, r, ok, rep = dynamics.relax_adaptive(s, 1e-10, 200000, check_every=20)
    assert ok
    assert np.abs(s.U.reshape(-1) - U_exact).max() <= 1e-8 * np.abs(U_exact).max()
    # the estimate settles on the slowest mode and its critical damping
    assert rep["lambda"] == pytest.approx(lam[0], rel=0.02)
    assert rep["alpha"] == pytest.approx(2.0 * np.sqrt(lam[0]), rel=0.01)
    # faster than fixed damping a decade away from critical on either side
    for a in (0.1 * rep["alpha"], 10.0 * rep["alpha"]):
        fixed_steps, _, fixed_ok = solver(a).relax(1e-10, 4 * steps, check_every=20)
        assert not fixed_ok or fixed_steps > 2 * steps


def _tangent_spectrum(p, U):
    """Eigenvalues of M^-1 K over the free DOFs, K by central differences of
    the oracle's internal force at U."""
    model = dynamics.Model.from_problem(p)
    free = np.ones(3 * p.n_nodes, dtype=bool)
    free[p.bc_dof] = False
    f = np.flatnonzero(free)
    h = 1e-7
    K = np.zeros((len(f), len(f)))
    for c, j in enumerate(f):
        Up = U.reshape(-1).copy()
        Um = Up.copy()
        Up[j] += h
        Um[j] -= h
        dF = (model.internal_forces(Up.reshape(-1, 3)) - model.internal_forces(Um.reshape(-1, 3)))
        K[:, c] = dF.reshape(-1)[f] / (2 * h)
    K = 0.5 * (K + K.T)
    return eigh(K, np.diag(np.repeat(model.mass, 3)[f]), eigvals_only=True)


def test_adaptive_relaxation_of_the_fe_cube():
    p = W.cube_compression_tet4(n=3, n_steps=200, strain=-0.1)
    plain = dynamics.ExplicitSolver.from_problem(p, alpha=5.0)
    steps_p, r_p, ok_p = plain.relax(1e-8, 60000, check_every=50)
    adapt = dynamics.ExplicitSolver.from_problem(p, alpha=5.0)
    steps_a, r_a, ok_a, rep = dynamics.relax_adaptive(adapt, 1e-8, 60000, check_every=50)
    assert ok_p and ok_a
    assert steps_a < steps_p
    # same equilibrium
    assert np.abs(adapt.U - plain.U).max() <= 1e-5 * np.abs(plain.U).max()
    # the converged quotient is an eigenvalue of the tangent problem: the
    # lowest one that the load excites (here the second: the lowest mode is
    # orthogonal to the symmetric compression and never enters D)
    lam = _tangent_spectrum(p, adapt.U)
    j = int(np.argmin(np.abs(lam - rep["lambda"]) / lam))
    assert j <= 2
    assert rep["lambda"] == pytest.approx(lam[j], rel=1e-3)
    assert rep["lambda"] >= lam[0] * (1 - 1e-6)
    assert rep["err_est"] < np.inf and rep["n_estimates"] > 0
