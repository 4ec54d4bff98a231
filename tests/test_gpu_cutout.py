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
