"""Explicit dynamics around the oracle forces (FP64).

Equation of motion (Eq. 13):  M U'' + D U' + sum_e F^(e) = R, with lumped
(diagonal) mass M and mass-proportional damping D = alpha M.  Central
differences (Sec. 2.2; the paper points to a textbook for the scheme) give the
three-level update used here, written out from the difference quotients

  M (U^{n+1} - 2U^n + U^{n-1}) / dt^2 + alpha M (U^{n+1} - U^{n-1}) / (2 dt)
      = R - F(U^n)

  =>  U^{n+1} = a (R - F) + b U^n + c U^{n-1},
      a = 2 dt^2 / ((2 + alpha dt) m),  b = 4 / (2 + alpha dt),
      c = (alpha dt - 2) / (2 + alpha dt),

started from rest (U^0 = U^-1 = 0).  Prescribed DOFs are overwritten with
g(t_{n+1}) after the update; fixed DOFs are prescribed DOFs with target 0.

Readings (the paper is silent on these):
* lumped mass: m_i = sum over elements containing node i of rho 0V / n_e.
* critical step (Eq. 14): dt_crit = min_e L_e / c_e with c_e the fastest
  (dilatational) wave speed sqrt(M_e / rho_e) of the material linearised at
  rest, M_e the largest eigenvalue of its acoustic tensor over all directions:
  M_e = kappa + 4/3 mu_eff + 16/9 (eta_a + eta_b).  mu_eff = mu + 2 C01 is the
  small-strain shear modulus (Mooney-Rivlin).  A fibre family adds
  eta (dI4bar)^2 to the second variation of Psi at rest (Table 3: the term
  eta / 2 (I4bar - 1)^2 has zero slope there), with dI4bar = 2 H : (A - I/3) for
  a displacement gradient H (the J^-2/3 of the modified invariant removes the
  trace); its acoustic contribution 4 eta ((A - I/3) n)^2 is largest along the
  fibre, 4 eta (2/3)^2 = 16/9 eta.  So M_e is exact for NH, MR and TI, and for
  OT an upper bound (exact when the two fibres coincide).  L_e is the
  length that makes Eq. 14 the central-difference limit 2 / omega_e of the
  element's highest frequency under lumped mass, bounded as for uniform-strain
  elements: omega_e^2 <= n_e c_e^2 sum_{i,a} 0B_ia^2 (+ n_e k lmax(Gamma Gamma^T)
  / (rho 0V) for the H8 hourglass stiffness, lmax by Gershgorin), so
  L_e = 2 / sqrt(n_e sum 0B^2 (+ hourglass term / c_e^2)).  For a cube of side h
  this is h / sqrt(6) (Kuhn tet) and 2h / sqrt(13.2) (brick, kappa_hg = 0.1).
  The edge-length style choices (smallest altitude, 0V / A_max) exceed the
  stable step of free boundary nodes and are not used.
* ramp: s(tau) = tau (Sec. 5.1) or the C2 quintic 10 tau^3 - 15 tau^4 + 6 tau^5,
  tau = min((n + 1) / ramp_steps, 1); ramp_steps <= 0 means s = 1.
* residual for dynamic relaxation: r = ||F - R|| over free DOFs divided by
  ||F - R|| over prescribed DOFs (the reaction), or the numerator alone when
  the reaction is zero.
* relaxation (Sec. 6 names dynamic relaxation only): the same damped step,
  checked every k steps on the force of the current state; a checked state
  counts only once its prescribed values have reached their targets (step
  index >= ramp_steps), since a slow ramp is quasi-static and has small
  residuals on the way; on success the update of that step is kept, so the
  returned state is one step past the checked one.
"""
import numpy as np

from . import anp, djtled, elements, hourglass, tled

TET4, HEX8 = elements.TET4, elements.HEX8


def lumped_mass(V0, rho, conn, n_nodes):
    n_e = conn.shape[1]
    m = np.zeros(n_nodes)
    np.add.at(m, conn.ravel(), np.repeat(rho * V0 / n_e, n_e))
    return m


def wave_modulus(mat):
    model = np.asarray(mat["model"])
    mu_eff = mat["mu"] + np.where(model == djtled.MR, 2.0 * mat["c01"], 0.0)
    fib = np.where((model == djtled.TI) | (model == djtled.OT), mat["eta_a"], 0.0) \
        + np.where(model == djtled.OT, mat["eta_b"], 0.0)
    return mat["kappa"] + 4.0 / 3.0 * mu_eff + 16.0 / 9.0 * fib


def critical_time_step(X, conn, elem_type, mat, V0, gamma=None, k_hg=None):
    """dt_crit = min_e L_e / c_e  (Eq. 14), L_e as in the module docstring."""
    J0 = elements.reference_jacobian(X, conn, elem_type)
    Hxi = elements.Hxi(elem_type)
    B0 = np.linalg.solve(J0, np.broadcast_to(Hxi, (J0.shape[0],) + Hxi.shape))
    n_e = conn.shape[1]
    c2 = wave_modulus(mat) / mat["rho"]
    w2 = n_e * c2 * np.einsum("eia,eia->e", B0, B0)
    if gamma is not None:
        gram = np.einsum("eqa,epa->eqp", gamma, gamma)
        lmax = np.max(np.abs(gram).sum(axis=2), axis=1)
        w2 = w2 + n_e * k_hg * lmax / (mat["rho"] * V0)
    return float(np.min(2.0 / np.sqrt(w2)))


def ramp(tau, kind):
    tau = np.clip(tau, 0.0, 1.0)
    if kind == 0:
        return tau
    return tau ** 3 * (10.0 - 15.0 * tau + 6.0 * tau ** 2)


class Model:
    """Mesh + material + precomputed oracle constants; evaluates F_int(U)."""

    def __init__(self, elem_type, X, conn, mat, a_dir=None, b_dir=None, hg_coeff=0.1,
                 R=None, anp=False, formulation="djtled"):
        """formulation: "djtled" (O-A, the paper's Jacobian-operator forces,
        Table 3) or "tled" (O-B, classical TLED through the deformation
        gradient and the second Piola-Kirchhoff stress, Eq. 4 and 54-55): the
        same discretisation, so both give the same trajectory up to rounding
        (the paper's Fig. 4 compares the two)."""
        if formulation not in ("djtled", "tled"):
            raise ValueError(formulation)
        self.formulation = formulation
        self.elem_type = int(elem_type)
        self.anp = bool(anp)
        if self.anp and formulation != "djtled":
            raise ValueError("average nodal pressure is built on the DJ-TLED forces")
        if self.anp and self.elem_type != TET4:
            raise ValueError("average nodal pressure is built for T4 meshes")
        self.X = np.asarray(X, dtype=np.float64)
        self.conn = np.asarray(conn, dtype=np.int64)
        self.mat = {k: (np.asarray(v, dtype=np.float64) if k != "model" else np.asarray(v))
                    for k, v in mat.items()}
        self.a_dir, self.b_dir = a_dir, b_dir
        with_mr = bool(np.any(self.mat["model"] == djtled.MR))
        self.pre = djtled.precompute(self.X, self.conn, self.elem_type, a_dir, b_dir,
                                     with_mr=with_mr)
        self.N = self.X.shape[0]
        self.R = np.zeros((self.N, 3)) if R is None else np.asarray(R, dtype=np.float64)
        if self.elem_type == HEX8:
            self.gamma, self.k_hg = hourglass.hourglass_constants(
                self.X, self.conn, self.mat["mu"], self.mat["kappa"], hg_coeff)
        self.mass = lumped_mass(self.pre["V0"], self.mat["rho"], self.conn, self.N)

    @classmethod
    def from_problem(cls, p, R=None, formulation="djtled"):
        mat = dict(model=p.model, mu=p.mu, kappa=p.kappa, rho=p.rho, eta_a=p.eta_a,
                   eta_b=p.eta_b, c01=p.c01)
        return cls(p.elem_type, p.X, p.conn, mat, p.a_dir, p.b_dir, p.hg_coeff, R,
                   anp=getattr(p, "anp", False), formulation=formulation)

    def element_forces(self, U):
        u_e = U[self.conn]
        if self.formulation == "tled":
            F = tled.element_forces(u_e, self.X, self.conn, self.elem_type, self.mat, self.a_dir, self.b_dir)
            if self.elem_type == HEX8:
                F = F + hourglass.hourglass_forces(u_e, self.gamma, self.k_hg)
            return F
        pbar = None
        if self.anp:
            J = djtled.kinematics(u_e, self.pre)["J"]
            pbar = anp.element_pressure(J, self.pre["V0"], self.mat["kappa"], self.conn, self.N)
        F = djtled.element_forces(u_e, self.pre, self.mat, pressure=pbar)
        if self.elem_type == HEX8:
            F = F + hourglass.hourglass_forces(u_e, self.gamma, self.k_hg)
        return F

    def internal_forces(self, U):
        """sum_e F^(e) (Eq. 13), added in ascending element id then local node."""
        F = np.zeros((self.N, 3))
        np.add.at(F, self.conn.ravel(), self.element_forces(U).reshape(-1, 3))
        return F

    def critical_time_step(self):
        if self.elem_type == HEX8:
            return critical_time_step(self.X, self.conn, self.elem_type, self.mat,
                                      self.pre["V0"], self.gamma, self.k_hg)
        return critical_time_step(self.X, self.conn, self.elem_type, self.mat, self.pre["V0"])


class ExplicitSolver:
    """Central-difference time stepping of a Model with prescribed DOFs."""

    def __init__(self, model: Model, bc_dof, bc_target, dt=None, dt_scale=0.9, alpha=0.0,
                 ramp_kind=1, ramp_steps=0):
        self.m = model
        self.dt = float(dt) if dt else dt_scale * model.critical_time_step()
        self.alpha = float(alpha)
        self.bc_dof = np.asarray(bc_dof, dtype=np.int64)
        self.bc_target = np.asarray(bc_target, dtype=np.float64)
        self.set_damping(self.alpha)
        self.ramp_kind, self.ramp_steps = int(ramp_kind), int(ramp_steps)
        self.free = np.ones(3 * model.N, dtype=bool)
        self.free[self.bc_dof] = False
        self.U = np.zeros((model.N, 3))
        self.U_prev = np.zeros((model.N, 3))
        self.n = 0

    def set_damping(self, alpha):
        """Coefficients a, b, c of the three-level update for damping alpha."""
        self.alpha = float(alpha)
        d = self.dt
        self.a = 2.0 * d * d / ((2.0 + self.alpha * d) * self.m.mass)
        self.b = 4.0 / (2.0 + self.alpha * d)
        self.c = (self.alpha * d - 2.0) / (2.0 + self.alpha * d)

    @classmethod
    def from_problem(cls, p, dt=None, alpha=None, R=None, formulation="djtled"):
        if dt is None and getattr(p, "dt", 0.0) > 0.0:
            dt = p.dt
        return cls(Model.from_problem(p, R, formulation), p.bc_dof, p.bc_target, dt=dt,
                   dt_scale=p.dt_scale, alpha=p.alpha if alpha is None else alpha,
                   ramp_kind=p.ramp_kind, ramp_steps=p.ramp_steps)

    def set_displacements(self, U0):
        """Warm start: U^0 = U^-1 = U0 (at rest)."""
        self.U = np.array(U0, dtype=np.float64).reshape(-1, 3)
        self.U_prev = self.U.copy()

    def prescribed(self, n_next):
        if self.ramp_steps > 0:
            s = ramp(n_next / self.ramp_steps, self.ramp_kind)
        else:
            s = 1.0
        return self.bc_target * s

    def residual(self, F):
        r = (F - self.m.R).ravel()
        num = np.linalg.norm(r[self.free])
        den = np.linalg.norm(r[~self.free])
        return float(num / den) if den > 0.0 else float(num)

    def step(self, return_force=False):
        F = self.m.internal_forces(self.U)
        U_next = self.a[:, None] * (self.m.R - F) + self.b * self.U + self.c * self.U_prev
        flat = U_next.reshape(-1)
        flat[self.bc_dof] = self.prescribed(self.n + 1)
        self.U_prev, self.U = self.U, flat.reshape(-1, 3)
        self.n += 1
        return F if return_force else None

    def run(self, n_steps):
        for _ in range(int(n_steps)):
            self.step()
        return self.U

    def relax(self, tol, max_steps, check_every=100):
        r = np.inf
        for i in range(int(max_steps)):
            n = self.n  # index of the state whose force is evaluated in this step
            check = (i + 1) % check_every == 0
            F = self.step(return_force=True)
            if check:
                r = self.residual(F)
                # a state counts only once its prescribed values are at the targets
                if r <= tol and n >= self.ramp_steps:
                    return i + 1, r, True
        return int(max_steps), r, False


# ---------------------------------------------------------------------------
# Adaptive dynamic relaxation
#
# Sec. 6 relaxes to equilibrium with dynamic relaxation and cites the adaptive
# form of the method without writing it out.  Reading used here (the published
# adaptive scheme, in these steps):
#   * the damped iteration converges fastest when the slowest mode is damped
#     critically, alpha = 2 omega_min, omega_min^2 = lambda_min(M^-1 K);
#   * late in the iteration the displacement change is dominated by the
#     slowest mode, so its Rayleigh quotient with the tangent stiffness
#     estimates lambda_min.  The change is taken over a whole check interval,
#     D = U^n - U^{n-k}, with K D ~ F(U^n) - F(U^{n-k}): over k steps the fast
#     modes' oscillations cancel, and the force difference stays well above
#     the rounding of single-precision forces near equilibrium;
#         lambda = D . (F(U^n) - F(U^{n-k})) / (D . M D)   over free DOFs;
#   * the changes then shrink by a fixed factor r per interval, and the
#     remaining distance to equilibrium is bounded by the geometric tail
#         |U* - U^n| <= r / (1 - r) |D|,  r = ||D_now|| / ||D_previous||,
#     the per-step rate being rho = r^(1/k).
# Estimates are taken at each check (every k steps) once the earlier state is
# past the ramp (prescribed values fixed between the two).

def rayleigh_quotient(D, dF, mass, free):
    """D . dF / (D . M D) over the free DOFs (D, dF: N x 3; mass: N)."""
    d = np.asarray(D, dtype=np.float64).reshape(-1)[free]
    f = np.asarray(dF, dtype=np.float64).reshape(-1)[free]
    m = np.repeat(np.asarray(mass, dtype=np.float64), 3)[free]
    den = float(np.dot(d * m, d))
    return float(np.dot(d, f)) / den if den > 0.0 else 0.0


def critical_damping(lam):
    """Mass-proportional damping that damps a mode of M^-1 K eigenvalue lam
    critically: alpha = 2 sqrt(lam)."""
    return 2.0 * float(np.sqrt(lam))


def interval_ratio(norm_now, norm_before):
    """Contraction of the displacement change from one interval to the next."""
    return float(norm_now / norm_before)


def error_estimate(r, d_max):
    """Geometric-tail bound r / (1 - r) |D| (inf when not contracting)."""
    return r / (1.0 - r) * d_max if r < 1.0 else np.inf


def relax_adaptive(solver, tol, max_steps, check_every=100, alpha_min=0.0, alpha_max=None,
                   disp_tol=0.0):
    """Dynamic relaxation of `solver` (an ExplicitSolver) with the damping
    re-estimated at every check.  Returns (steps, residual, converged, report)
    with report = {alpha, lambda, rho, err_est, n_estimates, alphas}."""
    k = int(check_every)
    assert k >= 1
    a_max = alpha_max if alpha_max and alpha_max > 0 else 2.0 / solver.dt
    free = solver.free
    rep = {"alpha": solver.alpha, "lambda": 0.0, "rho": 0.0, "err_est": np.inf, "n_estimates": 0,
           "alphas": []}
    norm_prev = 0.0
    snap = None                            # (step index, U, F) of the previous check
    r = np.inf
    for i in range(int(max_steps)):
        n = solver.n                       # state whose force this step evaluates
        U_n = solver.U.copy()
        F = solver.step(return_force=True)
        if (i + 1) % k == 0:
            r = solver.residual(F)
            past = snap is not None and (solver.ramp_steps <= 0 or snap[0] >= solver.ramp_steps)
            if past:
                D = U_n - snap[1]
                lam = rayleigh_quotient(D, F - snap[2], solver.m.mass, free)
                if lam > 0.0:
                    alpha = min(max(critical_damping(lam), alpha_min), a_max)
                    solver.set_damping(alpha)
                    rep["lambda"] = lam
                    rep["n_estimates"] += 1
                d = D.reshape(-1)[free]
                norm = float(np.linalg.norm(d))
                if norm_prev > 0.0 and norm > 0.0:
                    ratio = interval_ratio(norm, norm_prev)
                    rep["rho"] = ratio ** (1.0 / k)
                    rep["err_est"] = error_estimate(ratio, float(np.abs(d).max()))
                else:
                    rep["rho"], rep["err_est"] = 0.0, np.inf
                norm_prev = norm
            else:
                rep["rho"], rep["err_est"] = 0.0, np.inf
                norm_prev = 0.0
            rep["alpha"] = solver.alpha
            rep["alphas"].append(solver.alpha)
            snap = (n, U_n, F)
            if (r <= tol and n >= solver.ramp_steps
                    and (disp_tol <= 0.0 or rep["err_est"] <= disp_tol)):
                return i + 1, r, True, rep
    return int(max_steps), r, False, rep
