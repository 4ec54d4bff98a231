"""The verification model of Sec. 5.1 (cube with four circular cut-outs, fixed
back face, ramped extension of the front face) on the GPU against the FP64
oracle, for T4 and H8 meshes and all four material models (Table 3), at the
paper's time step dt = 5e-5 s."""
import numpy as np
import pytest

from oracle import dynamics
from paper_2106_14189_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DISP_TOL = 1e-4   # rel-Linf after N steps, FP32 stepping against FP64


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_14189_gb300 import binding
    return binding


@pytest.mark.parametrize("et", [W.TET4, W.HEX8])
@pytest.mark.parametrize("model", [W.NH, W.TI, W.OT, W.MR])
def test_cutout_cube_trajectory(B, et, model):
    # smallest of the six sizes (10 cells per side, 3.7e3 DOFs); the first 400
    # of the 20000 steps at the paper's ramp rate (0.05 m over 1 s)
    n_steps = 400
    p = W.cutout_cube(et, 10, model, n_steps=n_steps, extension=0.05 * n_steps / 20000)
    with B.Mesh(p) as m:
        assert abs(m.dt - 5e-5) < 1e-15
        m.run(n_steps)
        U = m.displacements()
    ref = dynamics.ExplicitSolver.from_problem(p).run(n_steps)
    err = np.abs(U - ref)
    assert err.max() <= DISP_TOL * np.abs(ref).max()
    # root-mean-square difference (Eq. 52 form), as reported for DJ-TLED vs TLED (Fig. 4)
    rmse = float(np.sqrt(np.mean(err ** 2)))
    print(f"cut-out cube {p.name}: rel-Linf {err.max() / np.abs(ref).max():.3e}, RMSE {rmse:.3e} m")
    assert rmse <= DISP_TOL * np.abs(ref).max()


def _procs():
    import os
    return max(1, min(16, os.cpu_count() or 1))


@pytest.mark.parametrize("et", [W.TET4, W.HEX8])
def test_cutout_cube_six_sizes_match_oracle(B, et):
    """All six sizes of Sec. 5.1 (10-34 cells per side, 3.7e3-1.06e5 DOFs), NH,
    the first 1000 of the 20000 steps at the paper's ramp rate: every DOF of
    the GPU trajectory against the FP64 oracle (run process-parallel over
    element blocks, oracle/parallel.py) within rel-Linf 1e-4."""
    from oracle.parallel import ParallelSolver
    n_steps = 1000
    for n in (10, 14, 18, 22, 28, 34):
        p = W.cutout_cube(et, n, W.NH, n_steps=n_steps, extension=0.05 * n_steps / 20000)
        with B.Mesh(p) as m:
            m.run(n_steps)
            U = m.displacements()
        with ParallelSolver(p, _procs()) as ps:
            ref = ps.run(n_steps)
        e = np.abs(U - ref).max() / np.abs(ref).max()
        print(f"cut-out cube T{et} n = {n} ({3 * p.n_nodes} DOFs): rel-Linf {e:.2e} after {n_steps} steps")
        assert e < DISP_TOL, (n, e)


@pytest.mark.parametrize("et", [W.TET4, W.HEX8])
def test_cutout_cube_full_run_against_classical_tled(B, et):
    """The smallest cut-out cube over the paper's whole run (20000 steps of
    5e-5 s, front face pulled 0.05 m), the GPU's DJ-TLED against the FP64
    classical TLED (deformation gradient, second Piola-Kirchhoff stress;
    Eq. 4, 54-55): the difference the paper plots as RMSE over time (Fig. 4),
    here checked every 2000 steps within rel-Linf 1e-4."""
    from oracle.parallel import ParallelSolver
    p = W.cutout_cube(et, 10, W.NH)
    rows = []
    with B.Mesh(p) as m, ParallelSolver(p, _procs(), formulation="tled") as ps:
        for k in range(10):
            m.run(2000)
            ref = ps.run(2000)
            U = m.displacements()
            err = np.abs(U - ref)
            rmse = float(np.sqrt(np.mean(err ** 2)))  # Eq. 52
            rows.append((2000 * (k + 1), err.max() / np.abs(ref).max(), rmse))
            assert err.max() < DISP_TOL * np.abs(ref).max(), rows[-1]
    print(f"T{et} n = 10, DJ-TLED (GPU, FP32) vs classical TLED (FP64): " +
          ", ".join(f"t = {s * 5e-5:.1f} s: RMSE {r:.2e} m" for s, _, r in rows))
