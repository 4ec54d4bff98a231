"""Average nodal pressure (T4) on the GPU against the oracle (oracle/anp.py).

Tolerances as in test_gpu_parity: forces within 1e-4 of the largest force,
trajectories within 1e-4 rel-Linf; the relaxed cantilever's tip deflection
within 1 % of the oracle's linear static solution (the load is small enough
that the geometric nonlinearity stays below that).
"""
import numpy as np
import pytest

from oracle import dynamics
from paper_2106_14189_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_14189_gb300 import binding
    return binding


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("model", [W.NH, W.TI, W.OT, W.MR])
@pytest.mark.parametrize("prec,tile", [(0, 256), (0, 64), (1, 128)])
def test_anp_forces_match_oracle(B, model, prec, tile):
    p = W.random_tet_mesh_problem(6000, seed=11, model=model)
    rng = np.random.default_rng(3)
    p.kappa = p.mu * rng.uniform(10.0, 60.0, size=p.n_elems)   # bulk moduli that differ
    p.anp = True
    U = rng.normal(size=(p.n_nodes, 3)) * 0.004   # strains of a few percent, no inversion
    ref = dynamics.Model.from_problem(p).internal_forces(U)
    with B.Mesh(p, precision=prec, tile_size=tile) as m:
        F = m.internal_forces(U)
    err = np.abs(F - ref).max() / np.abs(ref).max()
    print(f"model {model} precision {prec} tile {tile}: {err:.2e}")
    assert err <= 1e-4


def test_anp_differs_from_element_pressure(B):
    """Under a non-homogeneous deformation ANP and the element form differ (the
    GPU path really averages), by the amount the oracle predicts."""
    p = W.random_tet_mesh_problem(3000, seed=4)
    U = np.random.default_rng(5).normal(size=(p.n_nodes, 3)) * 0.004
    with B.Mesh(p, assembly=2) as m:
        F_el = m.internal_forces(U)
    p.anp = True
    with B.Mesh(p) as m:
        F_anp = m.internal_forces(U)
    ref_anp = dynamics.Model.from_problem(p).internal_forces(U)
    p.anp = False
    ref_el = dynamics.Model.from_problem(p).internal_forces(U)
    d_gpu, d_ref = F_anp - F_el, ref_anp - ref_el
    assert np.abs(d_ref).max() > 0.05 * np.abs(ref_el).max()
    assert np.abs(d_gpu - d_ref).max() <= 2e-4 * np.abs(ref_el).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_anp_trajectory_matches_oracle(B, prec):
    p = W.cube_compression_tet4(n=6, n_steps=400, strain=-0.1)
    p.anp = True
    with B.Mesh(p, precision=prec) as m:
        m.run(400)
        U = m.displacements()
        dt = m.dt
    s = dynamics.ExplicitSolver.from_problem(p, dt=dt)
    U_ref = s.run(400)
    err = rel_linf(U, U_ref)
    print(f"precision {prec}: rel-Linf {err:.2e}")
    assert err <= 1e-4


def _cantilever(anp, nu=0.49):
    X, conn = W.box_tet4(20, 2, 2, 1.0, 0.1, 0.1)
    mu, kappa = W.lame_from_E_nu(3000.0, nu)
    E = conn.shape[0]
    clamped = np.flatnonzero(X[:, 0] < 1e-9)
    tip = np.flatnonzero(X[:, 0] > 1.0 - 1e-9)
    bc = np.concatenate([3 * clamped, 3 * clamped + 1, 3 * clamped + 2])
    p = W.Problem(name="cantilever", elem_type=W.TET4, X=X, conn=conn,
                  model=np.zeros(E, dtype=np.uint8), mu=np.full(E, mu), kappa=np.full(E, kappa),
                  rho=np.full(E, 1000.0), eta_a=np.zeros(E), eta_b=np.zeros(E), c01=np.zeros(E),
                  a_dir=np.tile([1.0, 0.0, 0.0], (E, 1)), b_dir=np.tile([0.0, 1.0, 0.0], (E, 1)),
                  bc_dof=bc, bc_target=np.zeros(len(bc)), anp=anp)
    R = np.zeros((X.shape[0], 3))
    R[tip, 2] = 1e-4 / len(tip)
    return p, R, tip


def _linear_tip(p, R, tip):
    """Oracle: stiffness at U = 0 by central differences, direct solve."""
    m = dynamics.Model.from_problem(p)
    N = p.n_nodes
    free = np.ones(3 * N, dtype=bool)
    free[p.bc_dof] = False
    f = np.flatnonzero(free)
    h = 1e-7
    K = np.zeros((len(f), len(f)))
    for c, j in enumerate(f):
        Up = np.zeros(3 * N)
        Up[j] = h
        dF = m.internal_forces(Up.reshape(-1, 3)) - m.internal_forces(-Up.reshape(-1, 3))
        K[:, c] = dF.reshape(-1)[f] / (2 * h)
    u = np.zeros(3 * N)
    u[f] = np.linalg.solve(K, R.reshape(-1)[f])
    return float(u.reshape(-1, 3)[tip, 2].mean())


def test_anp_cantilever_relaxes_to_the_oracle_solution(B):
    """Dynamic relaxation of the loaded cantilever (adaptive damping,
    compensated precision): with ANP the tip deflection is several times the
    locked element formulation's, and each equals the oracle's static one."""
    out = {}
    for anp in (False, True):
        p, R, tip = _cantilever(anp)
        ref = _linear_tip(p, R, tip)
        with B.Mesh(p, precompute=False, precision=1, relax_check_every=100, assembly=2) as m:
            B.dj_mesh_set_loads(m.h, R)
            m.dt = B.dj_precompute(m.h, m.params)
            st, steps, r, rep = m.relax_adaptive(1e-5, 400_000)
            tip_gpu = float(m.displacements()[tip, 2].mean())
        print(f"anp {anp}: tip {tip_gpu:.4e} (oracle {ref:.4e}), {steps} steps, alpha {rep['alpha']:.3f}")
        assert st == 0
        assert tip_gpu == pytest.approx(ref, rel=1e-2)
        out[anp] = tip_gpu
    assert out[True] > 4 * out[False]


def test_anp_argument_checks(B):
    p = W.cube_shear(W.HEX8, 3)
    p.anp = True
    with pytest.raises(B.DJError):
        B.Mesh(p)
    q = W.cube_shear(W.TET4, 3)
    q.anp = True
    with pytest.raises(B.DJError):
        B.Mesh(q, assembly=1)


def test_anp_in_a_batch_matches_the_oracle(B):
    """T4 meshes with average nodal pressure stepped together in one batch
    (one graph) land on the oracle's trajectories."""
    probs = [W.cube_compression_tet4(n=n, n_steps=200, strain=-0.1) for n in (4, 5, 6)]
    for p in probs:
        p.anp = True
    with B.Batch(probs, anp=1, assembly=2) as bt:
        bt.run(200)
        Ub = [bt.displacements(i) for i in range(len(probs))]
        dts = [B.dj_batch_instance_info(bt.b, i)[2] for i in range(len(probs))]
    for p, U, dt in zip(probs, Ub, dts):
        ref = dynamics.ExplicitSolver.from_problem(p, dt=dt).run(200)
        assert rel_linf(U, ref) <= 1e-4
