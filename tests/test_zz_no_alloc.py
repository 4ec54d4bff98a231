"""dj_residual_norms_static: the relaxation residual for callers that cannot
allocate device memory (code inside another framework's memory pool, real-time
loops that must stay out of the allocator, plugins handed buffers by a host
application).  It reduces into a fixed device array of the library instead of
allocating, so it must give the residual of the regular path
(dj_evaluate_field) on consecutive calls that reuse that array.  This file is
named to be collected last."""
import numpy as np
import pytest

from paper_2106_14189_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-4  # the force tolerance of the parity tests


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_14189_gb300 import binding
    return torch, binding


def _case(torch, B, p, seed):
    """(residual from the static-scratch call, residual from dj_evaluate_field)."""
    rng = np.random.default_rng(seed)
    U = rng.normal(size=(p.n_nodes, 3)) * 0.003
    U.reshape(-1)[p.bc_dof] = p.bc_target  # prescribed DOFs at their targets
    with B.Mesh(p) as m:
        dU = torch.tensor(U.astype(np.float32).reshape(-1), device="cuda")
        r_ref, inverted = B.dj_evaluate_field(m.h, dU.data_ptr())
        assert not inverted
        F = m.internal_forces(U.astype(np.float32).astype(np.float64))
    pres = np.zeros(3 * p.n_nodes, dtype=np.uint8)
    pres[p.bc_dof] = 1
    dF = torch.tensor(F.astype(np.float32).reshape(-1), device="cuda")
    dP = torch.tensor(pres, device="cuda")
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    st = B.dj_residual_norms_static(dF.data_ptr(), dP.data_ptr(), p.n_nodes, out.data_ptr())
    assert st == 0
    torch.cuda.synchronize()
    num, den = out.cpu().numpy()
    return float(np.sqrt(num) / np.sqrt(den)), r_ref


def test_static_scratch_residual_matches_regular_path_on_consecutive_calls(env):
    torch, B = env
    # two calls in a row, the second on a smaller problem, so that the second
    # reads a scratch array still holding the first call's partial sums
    big = W.cube_shear(W.TET4, 14, n_steps=100)
    small = W.random_hex_mesh_problem(5, seed=3)
    for p, seed in ((big, 0), (small, 1)):
        r_static, r_ref = _case(torch, B, p, seed)
        assert np.isfinite(r_ref) and r_ref > 0
        assert abs(r_static - r_ref) <= TOL * r_ref, (p.name, r_static, r_ref)


def test_static_scratch_rejects_sizes_beyond_its_capacity(env):
    torch, B = env
    dF = torch.zeros(3, device="cuda")
    dP = torch.zeros(3, dtype=torch.uint8, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert B.dj_residual_norms_static(dF.data_ptr(), dP.data_ptr(), 65536 * 256 + 1, out.data_ptr()) == 9
    assert B.dj_residual_norms_static(dF.data_ptr(), dP.data_ptr(), 0, out.data_ptr()) == 1
