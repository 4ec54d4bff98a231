"""GPU parity of the DJ-TLED step (CUDA library through the C ABI) against the
FP64 oracle.

Tolerances (stated once, used everywhere below):
* forces:        max |F_gpu - F_ref| <= 1e-4 max |F_ref|   (FP32 element arithmetic)
* displacements: rel-Linf = max |U_gpu - U_ref| / max |U_ref| <= 1e-4 after N steps
  (the tolerance the build targets for FP32 against FP64).
"""
import numpy as np
import pytest

from oracle import dynamics
from paper_2106_14189_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4
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


MODELS = [W.NH, W.TI, W.OT, W.MR]


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("renumber,assembly,tile,prec", [(1, 1, 0, 0), (0, 1, 96, 0), (1, 0, 0, 0),
                                                         (0, 0, 0, 0), (1, 1, 512, 0), (1, 1, 32, 0),
                                                         (1, 1, 0, 1), (1, 0, 0, 1), (1, 2, 0, 0),
                                                         (1, 2, 64, 1), (0, 2, 160, 0), (1, 1, 32, 1)])
def test_tet4_forces_match_oracle(B, model, renumber, assembly, tile, prec):
    # 6 * 7^3 = 2058 elements: several tiles plus a ragged tail
    p = W.random_tet_mesh_problem(2058, seed=11 + model, model=model)
    rng = np.random.default_rng(5)
    # nodal noise of 0.5 % of the box size: strains of a few percent, no inversion
    U = rng.normal(size=(p.n_nodes, 3)) * 0.005
    with B.Mesh(p, renumber=renumber, assembly=assembly, tile_size=tile, precision=prec) as m:
        F = m.internal_forces(U)
    ref = dynamics.Model.from_problem(p).internal_forces(U)
    assert rel_linf(F, ref) < FORCE_TOL


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("assembly,tile,prec", [(1, 0, 0), (0, 0, 0), (1, 256, 0), (1, 64, 0),
                                                (1, 0, 1), (0, 0, 1), (2, 0, 0), (2, 256, 1),
                                                (1, 32, 0), (1, 32, 1)])
def test_hex8_forces_match_oracle(B, model, assembly, tile, prec):
    p = W.random_hex_mesh_problem(9, seed=21 + model, model=model)  # 729 bricks, ragged
    p.hg_coeff = 0.15
    rng = np.random.default_rng(6)
    U = rng.normal(size=(p.n_nodes, 3)) * 0.004
    with B.Mesh(p, assembly=assembly, tile_size=tile, precision=prec) as m:
        F = m.internal_forces(U)
    ref = dynamics.Model.from_problem(p).internal_forces(U)
    assert rel_linf(F, ref) < FORCE_TOL


@pytest.mark.parametrize("et", [4, 8])
def test_single_element_mesh(B, et):
    X, conn = W.single_element(et, seed=4)
    E = 1
    mat = dict(model=np.full(E, W.TI, dtype=np.uint8), mu=np.full(E, 1000.0),
               kappa=np.full(E, 30000.0), rho=np.full(E, 1000.0), eta_a=np.full(E, 2000.0),
               eta_b=np.zeros(E), c01=np.zeros(E), a_dir=np.array([[1.0, 2.0, 0.5]]),
               b_dir=np.array([[0.0, 1.0, 0.0]]))
    p = W.Problem(name="one", elem_type=et, X=X, conn=conn, bc_dof=np.array([0, 1, 2], dtype=np.int64),
                  bc_target=np.array([0.0, 0.0, 0.05]), ramp_steps=50, **mat)
    with B.Mesh(p) as m:
        m.run(120)
        U = m.displacements()
    ref = dynamics.ExplicitSolver.from_problem(p).run(120)
    assert rel_linf(U, ref) < DISP_TOL


@pytest.fixture(scope="module")
def cfg1_reference():
    p = W.cube_compression_tet4(10, 2000)
    s = dynamics.ExplicitSolver.from_problem(p)
    out = {}
    for n in (500, 2000):
        s.run(n - s.n)
        out[n] = s.U.copy()
    return p, s.dt, out


def test_cfg1_trajectory_2000_steps(B, cfg1_reference):
    """Tet4 cube 10^3 x 6 (6000 T4), NH, E = 3 kPa, nu = 0.49, -20 % z on a smooth ramp."""
    p, dt_ref, ref = cfg1_reference
    with B.Mesh(p) as m:
        assert abs(m.dt - dt_ref) < 1e-12 * dt_ref
        m.run(500)
        U500 = m.displacements()
        m.run(1500)
        U2000 = m.displacements()
        info = m.info()
    assert info.step == 2000
    assert rel_linf(U500, ref[500]) < DISP_TOL
    e = rel_linf(U2000, ref[2000])
    rmse = float(np.sqrt(np.mean((U2000 - ref[2000]) ** 2)))  # Eq. 52
    print(f"cfg1 rel-Linf {e:.3e} RMSE {rmse:.3e} m")
    assert e < DISP_TOL


def test_hex8_trajectory_shear(B):
    p = W.cube_shear(W.HEX8, 8, n_steps=1500, shear=0.1)
    with B.Mesh(p) as m:
        m.run(1500)
        U = m.displacements()
        dt = m.dt
    s = dynamics.ExplicitSolver.from_problem(p)
    assert abs(s.dt - dt) < 1e-12 * dt
    ref = s.run(1500)
    e = rel_linf(U, ref)
    print(f"hex8 cube 8 shear 1500 steps rel-Linf {e:.3e}")
    assert e < DISP_TOL


def test_anisotropic_ellipsoid_damped(B):
    # coarse (7 mm) version of the brain-sized ellipsoid: surface patches cover only a
    # few nodes, so the patch displacements are scaled down to keep elements valid
    p = W.ellipsoid_tet4(h=7e-3, seed=3, disp_range=(1e-3, 3e-3))
    p.alpha = 5.0
    p.ramp_steps = 500
    with B.Mesh(p) as m:
        m.run(700)
        U = m.displacements()
    ref = dynamics.ExplicitSolver.from_problem(p).run(700)
    e = rel_linf(U, ref)
    print(f"ellipsoid (7 mm, TI) 700 steps rel-Linf {e:.3e}")
    assert e < DISP_TOL


def test_orthotropic_and_mooney_rivlin_trajectories(B):
    for model in (W.OT, W.MR):
        p = W.random_tet_mesh_problem(750, seed=40 + model, model=model)
        p.ramp_steps = 300
        p.alpha = 2.0
        with B.Mesh(p) as m:
            m.run(400)
            U = m.displacements()
        ref = dynamics.ExplicitSolver.from_problem(p).run(400)
        assert rel_linf(U, ref) < DISP_TOL, model


def test_external_loads(B):
    p = W.random_hex_mesh_problem(4, seed=8)
    p.ramp_steps = 100
    rng = np.random.default_rng(1)
    R = rng.normal(size=(p.n_nodes, 3)) * 0.05
    m = B.Mesh(p, precompute=False)
    B.dj_mesh_set_loads(m.h, R)
    m.dt = B.dj_precompute(m.h, m.params)
    m.run(200)
    U = m.displacements()
    m.close()
    ref = dynamics.ExplicitSolver.from_problem(p, R=R).run(200)
    assert rel_linf(U, ref) < DISP_TOL


def test_deterministic_and_checkpoint_resume_bit_identical(B):
    p = W.cube_compression_tet4(6, 300)
    with B.Mesh(p) as a, B.Mesh(p) as b:
        a.run(300)
        b.run(150)
        blob = B.dj_get_state(b.h)
        b.run(150)
        Ua, Ub = a.displacements(), b.displacements()
        assert np.array_equal(Ua, Ub)
        B.dj_set_state(b.h, blob)
        assert B.dj_get_info(b.h).step == 150
        b.run(150)
        assert np.array_equal(b.displacements(), Ua)


@pytest.mark.parametrize("assembly", [1, 0])
def test_graph_and_direct_launch_agree(B, assembly):
    p = W.cube_shear(W.HEX8, 5, n_steps=100)
    with B.Mesh(p, assembly=assembly) as a, B.Mesh(p, assembly=assembly) as b:
        a.run(100)  # graph replays of 32 steps + 4 direct steps
        for _ in range(100):
            b.step()
        assert np.array_equal(a.displacements(), b.displacements())
        fa, fu = B.dj_run_n_profiled(b.h, 10)
        assert fa > 0 and fu > 0


@pytest.mark.parametrize("assembly", [2, 0])
def test_profile_kernels_leaves_the_trajectory_unchanged(B, assembly):
    import torch
    p = W.cube_shear(W.TET4, 6, n_steps=60)
    flush = torch.empty(8 << 20, dtype=torch.uint8, device="cuda")
    with B.Mesh(p, assembly=assembly) as a, B.Mesh(p, assembly=assembly) as b:
        a.run(30)
        b.run(30)
        tf, tu = B.dj_profile_kernels(b.h, 5, flush.data_ptr(), flush.numel())
        assert tf > 0 and tu > 0
        tf, tu = B.dj_profile_kernels(b.h, 3)
        assert tf > 0 and tu > 0
        a.run(30)
        b.run(30)
        assert np.array_equal(a.displacements(), b.displacements())


def test_inverted_reference_element_is_reported(B):
    X, conn = W.cube_tet4(3)
    conn = conn.copy()
    conn[17, [1, 2]] = conn[17, [2, 1]]
    p = W.cube_compression_tet4(3, 10)
    p.conn = conn
    with pytest.raises(B.DJError) as e:
        B.Mesh(p)
    assert e.value.status == 3 and "element 17" in str(e.value)


def test_inversion_while_stepping_is_reported(B):
    p = W.cube_compression_tet4(3, 10, strain=-3.0)   # crush to -300 % in 10 steps
    with B.Mesh(p) as m:
        m.run(40)
        with pytest.raises(B.DJError) as e:
            m.sync()
        assert e.value.status in (3, 5)
        # a new field starts a new trajectory with an empty error record
        B.dj_mesh_update_bc_targets(m.h, 0.01 * np.asarray(p.bc_target))
        m.set_displacements(np.zeros((p.n_nodes, 3)))
        B.dj_set_step(m.h, 0)
        m.run(5)
        m.sync()
        assert np.isfinite(m.displacements()).all()


def test_dt_above_critical_rejected(B):
    p = W.cube_compression_tet4(3, 10)
    with pytest.raises(B.DJError) as e:
        B.Mesh(p, dt=1.0)
    assert e.value.status == 1
    for bad_tile in (48, 1024):
        with pytest.raises(B.DJError) as e:
            B.Mesh(p, tile_size=bad_tile)
        assert e.value.status == 1


def test_slot_and_tile_assembly_trajectories_agree(B):
    p = W.cube_compression_tet4(8, 400)
    with B.Mesh(p, assembly=0) as a, B.Mesh(p, assembly=1) as b:
        a.run(400)
        b.run(400)
        Ua, Ub = a.displacements(), b.displacements()
    assert rel_linf(Ub, Ua) < 1e-5


@pytest.mark.parametrize("et", [4, 8])
@pytest.mark.parametrize("tile", [0, 32])
def test_tma_pipeline_equals_per_tile_blocks(B, et, tile):
    """Same tiles, same fixed summation order: the persistent bulk-copy pipeline
    and the one-block-per-tile kernel (one warp per tile at 32) give
    bit-identical trajectories."""
    p = W.cube_shear(et, 9 if et == 4 else 10, n_steps=300)
    with B.Mesh(p, assembly=1, tile_size=tile) as a, B.Mesh(p, assembly=2, tile_size=tile) as b:
        a.run(300)
        b.run(300)
        assert np.array_equal(a.displacements(), b.displacements())
        b.sync()


# The persistent bulk-copy kernel (assembly 2) walks tiles b, b + grid, ...:
# from the second tile of a block on, the stage ring is reused, the mbarrier
# phases flip and the node list of the next tile rides in the current stage.
# A grid cap (dj_params.max_blocks) makes every block walk several tiles on
# meshes small enough for the oracle.
STEADY = [(4, 0, 3), (4, 64, 4), (8, 0, 2), (8, 64, 3)]  # (element, tile size, blocks)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("model", [W.NH, W.TI, W.OT, W.MR])
@pytest.mark.parametrize("et,tile,blocks", STEADY)
def test_tma_steady_state_forces_match_oracle(B, et, tile, blocks, model, prec):
    """Bulk-copy pipeline with several tiles per block: every nodal force against
    the oracle within the force tolerance."""
    if et == 4:
        p = W.random_tet_mesh_problem(2058, seed=31 + model, model=model)
        U = np.random.default_rng(7).normal(size=(p.n_nodes, 3)) * 0.005
    else:
        p = W.random_hex_mesh_problem(9, seed=41 + model, model=model)
        p.hg_coeff = 0.15
        U = np.random.default_rng(8).normal(size=(p.n_nodes, 3)) * 0.004
    with B.Mesh(p, assembly=2, tile_size=tile, precision=prec, max_blocks=blocks) as m:
        info = m.info()
        F = m.internal_forces(U)
    assert info.grid == blocks and info.n_tiles >= 3 * info.grid, (info.grid, info.n_tiles)
    ref = dynamics.Model.from_problem(p).internal_forces(U)
    assert rel_linf(F, ref) < FORCE_TOL


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("model", [W.NH, W.TI])
@pytest.mark.parametrize("et,tile,blocks", STEADY)
def test_tma_steady_state_trajectory_matches_oracle(B, et, tile, blocks, model, prec):
    """Bulk-copy pipeline with several tiles per block, stepped: every DOF against
    the FP64 oracle's trajectory within rel-Linf 1e-4 (Algorithm 1 run-time loop,
    Eq. 13), and against the one-block-per-tile kernel (same tiles, same
    summation order): bit-identical where both kernels compile the element
    routine alike, else within 1e-6 (the compiler may contract a product and a
    sum into one FMA in one kernel and not in the other)."""
    if et == 4:
        p = W.random_tet_mesh_problem(4374, seed=51 + model, model=model)
    else:
        p = W.random_hex_mesh_problem(10, seed=61 + model, model=model)
    p.ramp_steps, p.alpha = 200, 2.0
    n = 300
    with B.Mesh(p, assembly=2, tile_size=tile, precision=prec, max_blocks=blocks) as m, \
            B.Mesh(p, assembly=1, tile_size=tile, precision=prec) as t:
        info = m.info()
        m.run(n)
        t.run(n)
        U, Ut = m.displacements(), t.displacements()
    assert info.grid == blocks and info.n_tiles >= 3 * info.grid, (info.grid, info.n_tiles)
    ref = dynamics.ExplicitSolver.from_problem(p).run(n)
    e = rel_linf(U, ref)
    d = rel_linf(U, Ut)
    print(f"steady-state bulk-copy T{et} model {model} prec {prec}: {info.n_tiles} tiles on "
          f"{info.grid} blocks, {n} steps, rel-Linf {e:.2e} (oracle), {d:.2e} (per-tile kernel)")
    assert e < DISP_TOL
    assert d < 1e-6


def test_relaxation_matches_oracle(B):
    """Plain FP32 stepping stalls near r ~ 1e-4 on this stiff (kappa / mu = 50) cube,
    so the tolerance here is 3e-4; the compensated mode reaches 1e-5 (below)."""
    p = W.cube_shear(W.HEX8, 4, shear=0.1)
    p.alpha, p.ramp_steps = 4.0, 200
    with B.Mesh(p, relax_check_every=50) as m:
        st, steps, r = m.relax(3e-4, 40000)
        U = m.displacements()
    s = dynamics.ExplicitSolver.from_problem(p)
    n_ref, r_ref, ok = s.relax(3e-4, 40000, check_every=50)
    assert ok and r <= 3e-4
    assert abs(steps - n_ref) <= 100
    assert rel_linf(U, s.U) < 1e-3


@pytest.mark.parametrize("et", [4, 8])
def test_compensated_relaxation_reaches_1e5(B, et):
    """Compensated precision relaxes the stiff cube to r <= 1e-5 and lands on the
    oracle's equilibrium."""
    p = W.cube_shear(et, 4 if et == 8 else 3, shear=0.1)
    p.alpha, p.ramp_steps = 4.0, 200
    with B.Mesh(p, relax_check_every=50, precision=1) as m:
        st, steps, r = m.relax(1e-5, 60000)
        U = m.displacements()
    s = dynamics.ExplicitSolver.from_problem(p)
    n_ref, r_ref, ok = s.relax(1e-5, 60000, check_every=50)
    assert ok and r <= 1e-5
    assert abs(steps - n_ref) <= 200
    assert rel_linf(U, s.U) < 2e-4


def test_compensated_small_strain_forces_are_accurate(B):
    """At 1e-4 strain the compensated force keeps the FP32 relative accuracy."""
    p = W.random_tet_mesh_problem(2058, seed=3)
    U = np.random.default_rng(9).normal(size=(p.n_nodes, 3)) * 2e-5
    ref = dynamics.Model.from_problem(p).internal_forces(U)
    with B.Mesh(p, precision=1) as m:
        F1 = m.internal_forces(U)
    assert rel_linf(F1, ref) < 2e-5


def test_cfg1_trajectory_compensated(B, cfg1_reference):
    p, dt_ref, ref = cfg1_reference
    with B.Mesh(p, precision=1) as m:
        m.run(2000)
        U = m.displacements()
    assert rel_linf(U, ref[2000]) < DISP_TOL


def test_full_size_cfg2b_sampled_nodes_bulk_copy_tiles_256(B):
    """1.23M-tet cube (59^3 x 6) in the benchmark's schedule (plain FP32, the
    persistent bulk-copy kernel with tiles of 256 on one wave of blocks, so every
    block walks several tiles): one update at sampled nodes against the oracle,
    which evaluates only
    their incident elements.  FP32 error model of the force at node i: 1e-4 of the
    largest incident element force, plus the volumetric term's absolute error
    kappa 0V |0B| dJ with dJ = 8 ulp(1) (J - 1 is formed as det(tJ) / det(0J) - 1)."""
    from oracle import tled
    p = W.cube_shear(W.TET4, 59, n_steps=5000)
    rng = np.random.default_rng(0)
    with B.Mesh(p, assembly=2, tile_size=256) as m:
        info = m.info()
        assert info.assembly == 2 and info.n_tiles > info.grid > 0, (info.n_tiles, info.grid)
        m.run(2000)
        U0 = m.displacements()
        m.step()
        U1 = m.displacements()
        m.step()
        U2 = m.displacements()
        dt = m.dt
    assert np.abs(U2).max() > 0
    sample = rng.choice(p.n_nodes, size=64, replace=False)
    checked = 0
    eps = float(np.finfo(np.float32).eps)
    for i in sample:
        els = np.nonzero((p.conn == i).any(axis=1))[0]
        sub = W.Problem(name="sub", elem_type=4, X=p.X, conn=p.conn[els], model=p.model[els],
                        mu=p.mu[els], kappa=p.kappa[els], rho=p.rho[els], eta_a=p.eta_a[els],
                        eta_b=p.eta_b[els], c01=p.c01[els], a_dir=p.a_dir[els], b_dir=p.b_dir[els],
                        bc_dof=np.zeros(0, dtype=np.int64), bc_target=np.zeros(0))
        mdl = dynamics.Model.from_problem(sub)
        Fe = mdl.element_forces(U1)
        F = mdl.internal_forces(U1)[i]
        B0, V0 = tled.shape_derivatives(p.X, p.conn[els], 4)
        vol_scale = np.sum(p.kappa[els] * V0 * np.abs(B0).max(axis=(1, 2)))
        a_i = 2 * dt * dt / (2 * mdl.mass[i])
        U2_ref = -a_i * F + 2 * U1[i] - U0[i]
        pres = np.isin(3 * i + np.arange(3), p.bc_dof)
        if pres.all():
            continue
        err = np.abs(U2[i] - U2_ref)[~pres].max()
        bound = a_i * (1e-4 * np.abs(Fe).max() + 8 * eps * vol_scale) \
            + 4 * np.spacing(np.float32(np.abs(U2[i]).max()))
        assert err <= bound, (i, err, bound)
        checked += 1
    assert checked > 40


@pytest.mark.parametrize("prec", [0, 1])
def test_displacements_into_pinned_and_pageable_buffers_agree(B, prec):
    """dj_get_displacements writes a page-locked buffer directly from its
    kernel and fills other host memory by a copy: both give the same values."""
    torch = pytest.importorskip("torch")
    p = W.cube_shear(W.TET4, 7, n_steps=100)
    with B.Mesh(p, precision=prec) as m:
        m.run(60)
        U_page = m.displacements()
        pinned = torch.empty((p.n_nodes, 3), dtype=torch.float64).pin_memory()
        U_pin = B.dj_get_displacements(m.h, p.n_nodes, out=pinned.numpy())
        assert np.array_equal(U_page, U_pin)
        assert np.abs(U_page).max() > 0


def _pinned_f64(torch, n, offset):
    """A float64 view of n values starting `offset` bytes into page-locked memory."""
    raw = torch.empty(8 * n + 8, dtype=torch.uint8).pin_memory()
    return raw, np.frombuffer(raw.numpy(), dtype=np.float64, count=n, offset=offset)


def test_per_step_targets_from_any_host_buffer_agree(B):
    """Prescribed targets changed before every step: a page-locked array (read
    by the scatter kernel through its device mapping), a misaligned view of
    page-locked memory and pageable memory (both staged on the host) give
    bit-identical trajectories, read back into the same three kinds of
    buffer; the moved DOFs sit on their last targets."""
    torch = pytest.importorskip("torch")
    p = W.cube_shear(W.TET4, 6, n_steps=40)
    base = np.asarray(p.bc_target, dtype=np.float64)
    nb, N = base.size, p.n_nodes
    out = {}
    for layout in ("pageable", "pinned", "pinned_misaligned"):
        keep = []
        if layout == "pageable":
            tgt, U = np.empty(nb), np.empty((N, 3))
        else:
            off = 0 if layout == "pinned" else 4
            r1, tgt = _pinned_f64(torch, nb, off)
            r2, u = _pinned_f64(torch, 3 * N, off)
            keep += [r1, r2]
            U = u.reshape(N, 3)
        with B.Mesh(p) as m:
            for k in range(30):
                tgt[:] = base * (0.5 + 0.02 * k) + 1e-4 * np.sin(k + np.arange(nb))
                B.dj_mesh_update_bc_targets(m.h, tgt)
                B.dj_step(m.h)
            B.dj_get_displacements(m.h, N, out=U)
        out[layout] = U.copy()
        last = tgt.copy()
    for layout in ("pinned", "pinned_misaligned"):
        assert np.array_equal(out[layout], out["pageable"]), layout
    # prescribed DOFs follow the ramp toward their targets: at step 30 of a
    # 40-step ramp each sits at ramp(30/40) times its last target (FP32)
    moved = np.abs(last) > 1e-3
    flat = out["pageable"].reshape(-1)[np.asarray(p.bc_dof)]
    ratio = flat[moved] / last[moved]
    assert np.ptp(ratio) < 1e-5 and 0.0 < ratio.mean() < 1.0


def test_brain_shift_configuration_matches_oracle(B):
    """Sec. 6's brain-shift setting at the paper's mesh size (28,770 T4 on the
    brain-sized ellipsoid; the paper's mesh has 28,764): neo-Hookean brain
    tissue, rho 1060, dt = 1.6e-4 s; 300 steps with the surface loads ramped
    over them, FP32 GPU against the FP64 oracle."""
    p = W.ellipsoid_tet4(h=5.35e-3, seed=0, patch_radius=0.025, disp_range=(0.5e-3, 2.5e-3), fibres=False)
    p.model[:] = W.NH
    p.mu[:], p.kappa[:], p.rho[:] = 1006.712, 50000.0, 1060.0
    p.eta_a[:], p.eta_b[:], p.c01[:] = 0.0, 0.0, 0.0
    p.dt, p.alpha, p.ramp_steps = 1.6e-4, 130.0, 300
    with B.Mesh(p) as m:
        m.run(300)
        U = m.displacements()
    ref = dynamics.ExplicitSolver.from_problem(p).run(300)
    err = rel_linf(U, ref)
    print(f"brain-shift setting, 300 steps: rel-Linf {err:.2e}")
    assert err < DISP_TOL


@pytest.mark.parametrize("assembly", [0, 1, 2])
def test_graph_programmatic_edges_bit_identical(B, assembly):
    """Graph replays with programmatic-launch edges between the steps give the
    same trajectory, bit for bit, as ordinary edges (and so does relaxation)."""
    p = W.cube_shear(W.TET4, 7, n_steps=200)
    p.alpha, p.ramp_steps = 40.0, 100
    out = []
    for pdl in (0, 1):
        with B.Mesh(p, assembly=assembly, graph_pdl=pdl, relax_check_every=50) as m:
            m.run(130)
            U = m.displacements()
            st, n, r = m.relax(1e-3, 3000, raise_on_fail=False)
            out.append((U, m.displacements(), n))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]


@pytest.mark.parametrize("prec", [1, 0])
def test_full_size_brain_ellipsoid_sampled_nodes(B, prec):
    """The 0.8M-T4 anisotropic brain-sized ellipsoid of the relaxation workload
    (h = 1.76 mm, two materials, TI fibres, six surface patches, alpha = 130 1/s,
    the schedule a mesh of this size gets by default) part way up its ramp: one
    damped update (Eq. 13) at 64 sampled free nodes against the oracle, which
    evaluates only their incident elements.  Error model of the FP32 force at a
    node as in the cube test: 1e-4 of the largest incident element force plus
    the volumetric term's rounding kappa 0V |0B| 8 ulp(1)."""
    from oracle import tled
    p = W.ellipsoid_tet4(h=1.76e-3, seed=0, patch_radius=0.025, disp_range=(0.5e-3, 2.5e-3))
    p.alpha, p.ramp_steps = 130.0, 2557
    p.bc_target = W.ellipsoid_load_case(p, 3)
    with B.Mesh(p, relax_check_every=50, precision=prec) as m:
        m.run(1200)
        U0 = m.displacements()
        m.step()
        U1 = m.displacements()
        m.step()
        U2 = m.displacements()
        dt = m.dt
        info = m.info()
    assert info.n_elems == p.n_elems and np.abs(U2).max() > 1e-4
    free = np.ones(3 * p.n_nodes, dtype=bool)
    free[p.bc_dof] = False
    cand = np.nonzero(free.reshape(-1, 3).all(axis=1) & (np.abs(U2).max(axis=1) > 1e-6))[0]
    sample = np.random.default_rng(1).choice(cand, size=64, replace=False)
    eps = float(np.finfo(np.float32).eps)
    ad = p.alpha * dt
    worst = 0.0
    for i in sample:
        els = np.nonzero((p.conn == i).any(axis=1))[0]
        sub = W.Problem(name="sub", elem_type=4, X=p.X, conn=p.conn[els], model=p.model[els],
                        mu=p.mu[els], kappa=p.kappa[els], rho=p.rho[els], eta_a=p.eta_a[els],
                        eta_b=p.eta_b[els], c01=p.c01[els], a_dir=p.a_dir[els], b_dir=p.b_dir[els],
                        bc_dof=np.zeros(0, dtype=np.int64), bc_target=np.zeros(0))
        mdl = dynamics.Model.from_problem(sub)
        Fe = mdl.element_forces(U1)
        F = mdl.internal_forces(U1)[i]
        B0, V0 = tled.shape_derivatives(p.X, p.conn[els], 4)
        vol_scale = np.sum(p.kappa[els] * V0 * np.abs(B0).max(axis=(1, 2)))
        a_i = 2 * dt * dt / ((2 + ad) * mdl.mass[i])
        U2_ref = -a_i * F + 4 / (2 + ad) * U1[i] + (ad - 2) / (2 + ad) * U0[i]
        err = np.abs(U2[i] - U2_ref).max()
        bound = a_i * (1e-4 * np.abs(Fe).max() + 8 * eps * vol_scale) \
            + 4 * np.spacing(np.float32(np.abs(U2[i]).max()))
        worst = max(worst, err / bound)
        assert err <= bound, (i, err, bound)
    print(f"brain ellipsoid 0.8M T4 TI, precision {prec}: worst error / bound {worst:.2f} over 64 nodes")


STEP_HOST_SCHEDULES = {  # name: (element, mesh options)
    "tiles": ("T4", dict(assembly=1)),
    "tiles-warp": ("T4", dict(assembly=1, tile_size=32)),
    "slots": ("T4", dict(assembly=0)),
    "bulk-copy": ("T4", dict(assembly=2, tile_size=256)),
    # one block of 256 threads for 294 targets: the force kernel's copy loops
    "bulk-copy-1-block": ("T4", dict(assembly=2, tile_size=256, max_blocks=1)),
    "bulk-copy-anp": ("T4", dict(assembly=2, tile_size=256, anp=1)),
    "hex-bulk-copy": ("H8", dict(assembly=2, tile_size=64)),
    "hex-slots": ("H8", dict(assembly=0)),
}


@pytest.mark.parametrize("sched", sorted(STEP_HOST_SCHEDULES))
@pytest.mark.parametrize("prec", [0, 1])
def test_step_host_matches_separate_calls(B, prec, sched):
    """dj_step_host (targets in, one step, displacements out, one
    synchronisation) gives bit for bit the trajectory of dj_mesh_update_bc_targets
    + dj_step + dj_get_displacements, with page-locked and pageable buffers, on
    every force schedule (each copies page-locked targets in its own way), and
    its FP32 output is the FP64 output rounded once; HostStep (the bound form)
    gives the same."""
    torch = pytest.importorskip("torch")
    elem, opts = STEP_HOST_SCHEDULES[sched]
    p = W.cube_shear(W.TET4, 6, n_steps=40) if elem == "T4" else W.cube_shear(W.HEX8, 6, n_steps=40)
    kw = dict(precision=prec, **opts)
    base = np.asarray(p.bc_target, dtype=np.float64)
    N = p.n_nodes
    ref, outs = [], {}
    with B.Mesh(p, **kw) as m:
        if sched == "bulk-copy-1-block":
            assert m.info().grid == 1 and base.size > 256
        assert m.info().assembly == opts["assembly"]
        for k in range(25):
            B.dj_mesh_update_bc_targets(m.h, base * (0.5 + 0.02 * k))
            B.dj_step(m.h)
            ref.append(m.displacements())
    for layout in ("pageable", "pinned"):
        if layout == "pinned":
            tgt = torch.empty(base.size, dtype=torch.float64).pin_memory().numpy()
            U64 = torch.empty((N, 3), dtype=torch.float64).pin_memory().numpy()
            U32 = torch.empty((N, 3), dtype=torch.float32).pin_memory().numpy()
            U64b = torch.empty((N, 3), dtype=torch.float64).pin_memory().numpy()
        else:
            tgt, U64, U32 = np.empty(base.size), np.empty((N, 3)), np.empty((N, 3), dtype=np.float32)
            U64b = np.empty((N, 3))
        with B.Mesh(p, **kw) as m, B.Mesh(p, **kw) as m2, B.Mesh(p, **kw) as m3, B.Mesh(p, **kw) as m4:
            step3 = B.HostStep(m3, tgt, U64b)
            for k in range(25):
                tgt[:] = base * (0.5 + 0.02 * k)
                B.dj_step_host(m.h, tgt, U64)
                B.dj_step_host(m2.h, tgt, U32)
                step3()
                B.dj_step_host(m4.h, tgt, None)  # no read-back
                assert np.array_equal(U64, ref[k]), (layout, k)
                assert np.array_equal(U32, U64.astype(np.float32)), (layout, k)
                assert np.array_equal(U64b, U64), (layout, k)
            assert np.array_equal(m4.displacements(), ref[-1]), layout
            assert m.info().step == m4.info().step == 25
            # the host's copy of the targets follows the device's (a new
            # precomputation starts from the last targets)
            B.dj_precompute(m.h, m.params)
            B.dj_step(m.h)
            B.dj_precompute(m2.h, m2.params)
            B.dj_mesh_update_bc_targets(m2.h, tgt)
            B.dj_step(m2.h)
            assert np.array_equal(m.displacements(), m2.displacements()), layout
        outs[layout] = U64.copy()
    assert np.abs(outs["pinned"]).max() > 0


def test_step_host_non_finite_pinned_target_is_not_applied(B):
    """A NaN among the targets (page-locked or pageable): the step runs with
    that DOF's previous target, the other targets are applied, and the call
    reports DJ_ERR_INVALID_ARG; the next call with finite targets succeeds."""
    torch = pytest.importorskip("torch")
    p = W.cube_shear(W.TET4, 4, n_steps=10)
    p.ramp_steps = 0
    base = np.asarray(p.bc_target, dtype=np.float64)
    moved = int(np.nonzero(np.abs(base) > 0)[0][0])
    tgt = torch.empty(base.size, dtype=torch.float64).pin_memory().numpy()
    U = np.empty((p.n_nodes, 3))
    with B.Mesh(p) as m:
        tgt[:] = base
        B.dj_step_host(m.h, tgt, U)
        before = U.reshape(-1)[p.bc_dof].copy()
        tgt[:] = 2 * base
        tgt[moved] = np.nan
        with pytest.raises(B.DJError) as e:
            B.dj_step_host(m.h, tgt, U)
        assert e.value.status == B.DJ_ERR_INVALID_ARG
        after = U.reshape(-1)[p.bc_dof]
        assert after[moved] == np.float32(before[moved])
        others = np.abs(base) > 0
        others[moved] = False
        assert np.allclose(after[others], 2 * base[others], rtol=1e-6)
        with pytest.raises(B.DJError):
            B.dj_step_host(m.h, np.full(base.size, np.nan), U)
        assert np.array_equal(U.reshape(-1)[p.bc_dof], after)  # nothing applied
        tgt[:] = 3 * base
        B.dj_step_host(m.h, tgt, U)
        assert np.allclose(U.reshape(-1)[p.bc_dof][np.abs(base) > 0], 3 * base[np.abs(base) > 0], rtol=1e-6)
