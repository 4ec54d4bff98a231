"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects bad input in host code before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2106_14189_gb300 import binding, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dj_tled.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return binding.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dj_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTS) == names


def test_params_default(lib):
    p = binding.default_params()
    assert p.dt_scale == 0.9 and p.hg_coeff == 0.1 and p.relax_check_every == 100
    assert p.renumber == 1 and p.ramp_kind == 1


def test_status_strings(lib):
    for s, name in binding.STATUS.items():
        assert binding.dj_status_string(s)
    assert binding.dj_status_string(3) == "inverted element"


def test_host_validation_errors(lib):
    X, conn = workloads.cube_tet4(2)
    with pytest.raises(binding.DJError) as e:
        binding.dj_mesh_create(5, X, conn)
    assert e.value.status == 1
    bad = conn.copy()
    bad[0, 0] = X.shape[0]
    with pytest.raises(binding.DJError) as e:
        binding.dj_mesh_create(4, X, bad)
    assert e.value.status == 2
    with pytest.raises(binding.DJError) as e:
        binding.dj_mesh_create(4, X, conn[:0])
    assert e.value.status == 2
    Xn = X.copy()
    Xn[3, 1] = np.nan
    with pytest.raises(binding.DJError) as e:
        binding.dj_mesh_create(4, Xn, conn)
    assert e.value.status == 1
    h = binding.dj_mesh_create(4, X, conn)
    try:
        E = conn.shape[0]
        ones = np.ones(E)
        with pytest.raises(binding.DJError) as e:
            binding.dj_mesh_set_materials(h, np.zeros(E), -ones, ones, ones)
        assert e.value.status == 1 and "mu" in binding.dj_last_error(h)
        with pytest.raises(binding.DJError) as e:
            binding.dj_mesh_set_materials(h, np.full(E, 7), ones, ones, ones)
        assert e.value.status == 1
        binding.dj_mesh_set_materials(h, np.zeros(E), ones, ones, ones)
        with pytest.raises(binding.DJError) as e:
            binding.dj_mesh_set_bcs(h, [0, 0], [0.0, 1.0])
        assert "duplicate" in binding.dj_last_error(h)
        with pytest.raises(binding.DJError):
            binding.dj_mesh_set_bcs(h, [3 * X.shape[0]], [0.0])
        binding.dj_mesh_set_bcs(h, [0, 1, 2], [0.0, 0.0, 0.1])
        with pytest.raises(binding.DJError) as e:
            binding.dj_step(h)
        assert e.value.status == 4
    finally:
        binding.dj_mesh_destroy(h)


def test_state_size_is_known_before_device_work(lib):
    X, conn = workloads.cube_hex8(2)
    h = binding.dj_mesh_create(8, X, conn)
    try:
        assert binding.dj_state_size(h) == 32 + 2 * 16 * X.shape[0]
        info = binding.dj_get_info(h)
        assert info.n_nodes == X.shape[0] and info.n_elems == conn.shape[0] and info.elem_type == 8
    finally:
        binding.dj_mesh_destroy(h)


@pytest.mark.parametrize("kind", ["random", "clustered", "degenerate"])
def test_symmetric_eigen_matches_numpy(lib, kind):
    """The host eigensolver behind the POD (cyclic Jacobi, no device work)
    against LAPACK's through numpy: eigenvalues to 1e-12 of the largest,
    orthonormal eigenvectors that satisfy A v = w v, and, inside a cluster of
    nearly equal eigenvalues, the same invariant subspace."""
    rng = np.random.default_rng({"random": 1, "clustered": 2, "degenerate": 3}[kind])
    n = 60
    Q = np.linalg.qr(rng.normal(size=(n, n)))[0]
    if kind == "random":
        lam = rng.uniform(0.1, 10.0, size=n)
    elif kind == "clustered":  # SPD, three tight clusters and a spread tail
        lam = np.concatenate([5.0 + 1e-9 * rng.normal(size=10), 2.0 + 1e-7 * rng.normal(size=15),
                              1.0 + 1e-12 * rng.normal(size=5), rng.uniform(1e-6, 0.5, size=30)])
    else:  # exactly repeated eigenvalues and a null space
        lam = np.concatenate([np.full(20, 3.0), np.full(20, 1.0), np.zeros(20)])
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    w, V = binding.dj_symmetric_eigen(A)
    w_ref, V_ref = np.linalg.eigh(A)
    assert np.all(np.diff(w) <= 0)
    assert np.abs(w - w_ref[::-1]).max() < 1e-12 * np.abs(w_ref).max()
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-12
    assert np.abs(A @ V - V * w).max() < 1e-12 * np.abs(w_ref).max()
    # clusters: projectors onto the eigenvectors of each group agree
    for lo, hi in [(4.0, 6.0), (1.5, 2.5), (0.9, 1.1), (2.9, 3.1)]:
        sel = (w > lo) & (w < hi)
        sel_ref = (w_ref > lo) & (w_ref < hi)
        assert sel.sum() == sel_ref.sum()
        if sel.any():
            P = V[:, sel] @ V[:, sel].T
            P_ref = V_ref[:, sel_ref] @ V_ref[:, sel_ref].T
            assert np.abs(P - P_ref).max() < 1e-6


def test_symmetric_eigen_rejects_bad_input(lib):
    A = np.eye(3)
    A[0, 1] = np.nan
    with pytest.raises(binding.DJError):
        binding.dj_symmetric_eigen(A)


class _FakeMesh:
    """Stands in for a Mesh in HostStep's host-side checks (no device)."""
    h = None

    def info(self):
        return type("Info", (), {"n_bc_dofs": 6, "n_nodes": 4})()


def test_host_step_checks_buffers_once(lib):
    """HostStep validates types, layout and sizes when it binds the buffers
    and keeps their addresses (the arrays are held)."""
    m = _FakeMesh()
    tgt, U = np.zeros(6), np.zeros((4, 3), dtype=np.float32)
    hs = binding.HostStep(m, tgt, U)
    assert hs._args[1] == tgt.ctypes.data and hs._args[2] == U.ctypes.data and hs._args[3] == 0
    assert binding.HostStep(m, tgt, np.zeros((4, 3)))._args[3] == 1
    assert binding.HostStep(m, None, None)._args[1:3] == (None, None)
    bad = [
        (np.zeros(5), U),                          # wrong number of targets
        (np.zeros(6, dtype=np.float32), U),        # targets not float64
        (np.zeros(12)[::2], U),                    # targets not contiguous
        (tgt, np.zeros((4, 2), dtype=np.float32)),  # wrong output size
        (tgt, np.zeros((4, 3), dtype=np.int32)),    # output neither float32 nor float64
        (tgt, np.zeros((3, 4)).T),                 # output not C-contiguous
    ]
    for t, u in bad:
        with pytest.raises(ValueError):
            binding.HostStep(m, t, u)


def test_host_address_cache_tells_reused_ids(lib):
    """The address cache of dj_step_host returns a buffer's own address, also
    after an earlier buffer with the same id has been freed."""
    for _ in range(50):
        a = np.zeros(1000)
        assert binding._host_addr(a) == a.ctypes.data
        assert binding._host_addr(a) == a.ctypes.data
        del a
    ro = np.zeros(8)
    ro.flags.writeable = False
    assert binding._host_addr(ro) == ro.ctypes.data
