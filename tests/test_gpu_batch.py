"""Batched solves: many independent meshes of uneven size advanced together.

Every instance of a batch must follow the same trajectory as the FP64 oracle
run on that instance alone (same per-instance time step), within the
displacement tolerance of the single-mesh tests (rel-Linf <= 1e-4).
"""
import numpy as np
import pytest

from oracle import dynamics
from paper_2106_14189_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DISP_TOL = 1e-4


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


def small_batch(n=6, seed=1, steps=300):
    probs = W.batch_instances(n, seed=seed, e_min=300, e_max=4000, n_steps=steps)
    return probs


def test_batch_instances_match_oracle(B):
    probs = small_batch()
    assert {p.elem_type for p in probs} == {4, 8}
    with B.Batch(probs) as bt:
        n_inst, n_nodes, n_elems, n_tet, n_hex = bt.info()
        assert n_inst == len(probs) and n_elems == sum(p.n_elems for p in probs)
        bt.run(300)
        bt.sync()
        for i, p in enumerate(probs):
            nn, ne, dt, _ = bt.instance_info(i)
            s = dynamics.ExplicitSolver.from_problem(p)
            assert nn == p.n_nodes and ne == p.n_elems
            assert abs(dt - s.dt) < 1e-12 * s.dt
            ref = s.run(300)
            assert rel_linf(bt.displacements(i), ref) < DISP_TOL, i


def test_batch_equals_single_meshes(B):
    probs = small_batch(4, seed=3, steps=200)
    with B.Batch(probs) as bt:
        bt.run(200)
        Ub = [bt.displacements(i) for i in range(len(probs))]
    for p, U in zip(probs, Ub):
        with B.Mesh(p) as m:
            m.run(200)
            assert rel_linf(U, m.displacements()) < 2e-5


def test_batch_relaxation_compensated_per_instance(B):
    probs = small_batch(4, seed=5, steps=1000)
    for p in probs:
        p.alpha = 6.0
    with B.Batch(probs, relax_check_every=50, precision=1) as bt:
        st, steps, r = bt.relax(1e-5, 80000)
        assert st == 0 and r <= 1e-5
        Ub = [bt.displacements(i) for i in range(len(probs))]
        rb = [bt.instance_info(i)[3] for i in range(len(probs))]
    assert max(rb) <= 1e-5
    # each instance relaxed alone on the GPU reaches the same equilibrium
    for i, p in enumerate(probs):
        with B.Mesh(p, relax_check_every=50, precision=1) as m:
            m.relax(1e-5, 80000)
            assert rel_linf(Ub[i], m.displacements()) < 2e-3, i
    # and the smallest one against the oracle
    i = int(np.argmin([p.n_elems for p in probs]))
    s = dynamics.ExplicitSolver.from_problem(probs[i])
    n, r_ref, ok = s.relax(1e-6, 200000, check_every=50)
    assert ok
    assert rel_linf(Ub[i], s.U) < 2e-3


def test_groups_must_not_share_nodes(B):
    X, conn = W.cube_tet4(2)
    h = B.dj_mesh_create(4, X, conn)
    try:
        grp = np.zeros(conn.shape[0], dtype=np.int32)
        grp[0] = 1
        with pytest.raises(B.DJError) as e:
            B.dj_mesh_set_groups(h, grp, 2)
        assert e.value.status == 1 and "shared" in B.dj_last_error(h)
    finally:
        B.dj_mesh_destroy(h)


def test_grouped_mesh_has_per_group_steps(B):
    pa = W.cube_compression_tet4(3, 50)
    pb = W.cube_compression_tet4(5, 50)
    X = np.concatenate([pa.X, pb.X + 3.0])
    conn = np.concatenate([pa.conn, pb.conn + pa.n_nodes])
    grp = np.concatenate([np.zeros(pa.n_elems, np.int32), np.ones(pb.n_elems, np.int32)])
    h = B.dj_mesh_create(4, X, conn)
    try:
        E = conn.shape[0]
        B.dj_mesh_set_materials(h, np.zeros(E), np.full(E, 1000.0), np.full(E, 40000.0),
                                np.full(E, 1000.0))
        B.dj_mesh_set_groups(h, grp, 2)
        B.dj_precompute(h, B.default_params())
        dt, dtc, _ = B.dj_get_group_info(h)
        assert dtc[0] > dtc[1] and abs(dtc[0] / dtc[1] - 5.0 / 3.0) < 1e-9
        assert np.allclose(dt, 0.9 * dtc)
    finally:
        B.dj_mesh_destroy(h)


def test_autotune_keeps_the_trajectory(B):
    """The autotuner times every schedule from the current state, keeps the
    fastest and restores the state: stepping on afterwards matches a mesh built
    with the chosen schedule from the start."""
    p = W.cube_shear(W.TET4, 12, n_steps=400)
    with B.Mesh(p) as m:
        m.run(200)
        chosen, ms = B.dj_autotune(m.h, steps=50)
        assert ms > 0 and chosen.assembly in (0, 1, 2)
        assert B.dj_get_info(m.h).step == 200
        m.run(200)
        U = m.displacements()
    with B.Mesh(p, assembly=chosen.assembly, tile_size=chosen.tile_size) as r:
        r.run(400)
        assert rel_linf(U, r.displacements()) < 1e-5


def test_cold_autotune_keeps_the_trajectory(B):
    import torch
    p = W.cube_shear(W.HEX8, 8, n_steps=300)
    flush = torch.empty(8 << 20, dtype=torch.uint8, device="cuda")
    with B.Mesh(p) as m:
        m.run(100)
        chosen, ms = B.dj_autotune_cold(m.h, 10, flush.data_ptr(), flush.numel())
        assert ms > 0 and chosen.assembly in (0, 1, 2)
        assert B.dj_get_info(m.h).step == 100
        m.run(200)
        U = m.displacements()
    with B.Mesh(p, assembly=chosen.assembly, tile_size=chosen.tile_size) as r:
        r.run(300)
        assert rel_linf(U, r.displacements()) < 1e-5


def test_batch_autotune(B):
    probs = small_batch(4, seed=7, steps=200)
    with B.Batch(probs) as bt:
        bt.run(100)
        B.dj_batch_autotune(bt.b, steps=20)
        bt.run(100)
        bt.sync()
        for i, p in enumerate(probs):
            ref = dynamics.ExplicitSolver.from_problem(p).run(200)
            assert rel_linf(bt.displacements(i), ref) < DISP_TOL


def test_benchmarked_batch_sampled_instances_match_oracle(B):
    """The benchmark's batch itself (256 seeded instances, 10.8M elements, T4 / H8,
    schedules chosen by dj_batch_autotune as the benchmark does): after 400
    steps, eight seeded instances among those the oracle steps in seconds
    (<= 20k elements) each match the FP64 oracle run on that instance alone
    within rel-Linf 1e-4."""
    probs = W.batch_instances(256, seed=0, n_steps=2000)
    n_steps = 400
    with B.Batch(probs) as bt:
        bt.run(20)
        bt.sync()
        B.dj_batch_autotune(bt.b, steps=20)
        # the autotuner restores the state it found; start the timed trajectory from rest
        for i in range(len(probs)):
            B.dj_batch_set_displacements(bt.b, i, np.zeros((probs[i].n_nodes, 3)))
        B.dj_batch_set_step(bt.b, 0)
        bt.run(n_steps)
        bt.sync()
        small = [i for i, p in enumerate(probs) if p.n_elems <= 20000]
        rng = np.random.default_rng(0)
        sample = sorted(rng.choice(small, size=8, replace=False))
        assert {probs[i].elem_type for i in sample} == {4, 8}
        for i in sample:
            p = probs[i]
            U = bt.displacements(i)
            ref = dynamics.ExplicitSolver.from_problem(p).run(n_steps)
            e = rel_linf(U, ref)
            print(f"batch instance {i} (T{p.elem_type}, {p.n_elems} elements): rel-Linf {e:.2e}")
            assert e < DISP_TOL, (i, e)
