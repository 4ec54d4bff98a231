"""Learned warm start: GPU kernels against the FP64 reference, and the gain of
the trained network over plain relaxation from rest."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_2106_14189_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_14189_gb300 import binding
    return torch, binding


def test_mlp_loss_and_gradients_match_reference(env):
    torch, B = env
    rng = np.random.default_rng(0)
    widths = [64, 256, 256, 256, 128]
    m = B.dj_mlp_create(widths, seed=3)
    try:
        n = B.dj_mlp_num_params(m)
        _, n_ref = ref.layout(widths)
        assert n == n_ref
        p = B.dj_mlp_get_params(m).astype(np.float64)
        X = rng.normal(size=(200, 64))
        T = rng.normal(size=(200, 128))
        w = rng.uniform(0.1, 3.0, size=128)
        dX = torch.tensor(X, dtype=torch.float32, device="cuda")
        dT = torch.tensor(T, dtype=torch.float32, device="cuda")
        dw = torch.tensor(w, dtype=torch.float32, device="cuda")
        loss = B.dj_mlp_loss_grad(m, dX.data_ptr(), dT.data_ptr(), dw.data_ptr(), 200)
        g = B.dj_mlp_get_grads(m).astype(np.float64)
        L_ref, g_ref = ref.loss_grad(p, widths, X, T, w)
        assert abs(loss - L_ref) < 1e-5 * L_ref
        assert np.abs(g - g_ref).max() < 1e-4 * np.abs(g_ref).max()
        dY = torch.empty((200, 128), device="cuda")
        B.dj_mlp_forward(m, dX.data_ptr(), 200, dY.data_ptr())
        Y_ref = ref.forward(p, widths, X)[-1]
        assert np.abs(dY.cpu().numpy() - Y_ref).max() < 1e-5 * np.abs(Y_ref).max()
        # one Adam step
        B.dj_mlp_adam_step(m, 1e-3)
        p1 = B.dj_mlp_get_params(m).astype(np.float64)
        p_ref, _, _ = ref.adam_step(p, g, np.zeros(n), np.zeros(n), 1, 1e-3)
        assert np.abs(p1 - p_ref).max() < 1e-6 + 1e-5 * np.abs(p_ref).max()
    finally:
        B.dj_mlp_destroy(m)


def test_training_reduces_loss(env):
    torch, B = env
    rng = np.random.default_rng(1)
    widths = [8, 32, 32, 4]
    X = rng.normal(size=(256, 8))
    T = np.tanh(X @ rng.normal(size=(8, 4)))
    m = B.dj_mlp_create(widths, seed=0)
    dX = torch.tensor(X, dtype=torch.float32, device="cuda")
    dT = torch.tensor(T, dtype=torch.float32, device="cuda")
    first = B.dj_mlp_loss_grad(m, dX.data_ptr(), dT.data_ptr(), 0, 256)
    for _ in range(500):
        B.dj_mlp_loss_grad(m, dX.data_ptr(), dT.data_ptr(), 0, 256, want_loss=False)
        B.dj_mlp_adam_step(m, 3e-3)
    last = B.dj_mlp_loss_grad(m, dX.data_ptr(), dT.data_ptr(), 0, 256)
    B.dj_mlp_destroy(m)
    assert last < 0.05 * first


def test_pod_matches_svd(env):
    torch, B = env
    rng = np.random.default_rng(2)
    rows, cols, r = 3000, 96, 12
    basis = np.linalg.qr(rng.normal(size=(rows, 20)))[0]
    Y = basis @ (rng.normal(size=(20, cols)) * np.geomspace(10, 0.01, 20)[:, None]) \
        + rng.normal(size=rows)[:, None]
    dY = torch.tensor(Y.T.copy(), dtype=torch.float32, device="cuda")  # snapshot-major
    mean = torch.empty(rows, device="cuda")
    modes = torch.empty((rows, r), device="cuda")
    sig = B.dj_pod_fit(dY.data_ptr(), rows, cols, r, mean.data_ptr(), modes.data_ptr())
    mean_ref, U_ref, s_ref = ref.pod(Y, r)
    assert np.abs(mean.cpu().numpy() - mean_ref).max() < 1e-5 * np.abs(mean_ref).max()
    assert np.allclose(sig, s_ref, rtol=1e-4)
    M = modes.cpu().numpy().astype(np.float64)
    assert np.abs(M.T @ M - np.eye(r)).max() < 1e-4
    # same subspace: projection of the reference modes onto the GPU modes
    assert np.abs(np.abs(np.diag(U_ref.T @ M)) - 1).max() < 1e-3
    # project / expand round trip of a snapshot in the span
    Q = torch.empty((cols, r), device="cuda")
    B.dj_pod_project(modes.data_ptr(), mean.data_ptr(), rows, r, dY.data_ptr(), cols, Q.data_ptr())
    R = torch.empty((cols, rows), device="cuda")
    B.dj_pod_expand(modes.data_ptr(), mean.data_ptr(), rows, r, Q.data_ptr(), cols, R.data_ptr())
    Yr = mean_ref[:, None] + U_ref @ (U_ref.T @ (Y - mean_ref[:, None]))
    assert np.abs(R.cpu().numpy().T - Yr).max() < 1e-4 * np.abs(Y).max()


def test_linear_fit_and_apply_match_reference(env):
    torch, B = env
    rng = np.random.default_rng(4)
    S, n_in, n_out = 300, 24, 40
    X = rng.normal(size=(S, n_in))
    X[:, -3:] = 0.0                      # switched-off inputs: ridge keeps the system solvable
    Y = X @ rng.normal(size=(n_in, n_out)) + 0.01 * rng.normal(size=(S, n_out))
    dX = torch.tensor(X, dtype=torch.float32, device="cuda")
    dY = torch.tensor(Y, dtype=torch.float32, device="cuda")
    dW = torch.empty((n_out, n_in), device="cuda")
    B.dj_linear_fit(dX.data_ptr(), dY.data_ptr(), S, n_in, n_out, 1e-6, dW.data_ptr())
    W_ref = ref.linear_fit(X, Y, 1e-6)
    W = dW.cpu().numpy().astype(np.float64)
    assert np.abs(W - W_ref).max() < 1e-4 * np.abs(W_ref).max()
    dZ = torch.ones((S, n_out), device="cuda")
    B.dj_linear_apply(dW.data_ptr(), n_out, n_in, dX.data_ptr(), S, -1.0, 2.0, dZ.data_ptr())
    Z_ref = 2.0 - X @ W.T
    assert np.abs(dZ.cpu().numpy() - Z_ref).max() < 1e-5 * np.abs(Z_ref).max()


def test_quadratic_features(env):
    torch, B = env
    rng = np.random.default_rng(5)
    S, ld, n = 37, 20, 7
    X = rng.normal(size=(S, ld))
    dX = torch.tensor(X, dtype=torch.float32, device="cuda")
    nf = n + n * (n + 1) // 2
    dF = torch.empty((S, nf), device="cuda")
    B.dj_quad_features(dX.data_ptr(), S, ld, n, dF.data_ptr())
    Xf = X.astype(np.float32).astype(np.float64)[:, :n]
    ref = np.hstack([Xf] + [Xf[:, i:i + 1] * Xf[:, i:] for i in range(n)])
    assert np.abs(dF.cpu().numpy() - ref).max() < 1e-6 * np.abs(ref).max()


def test_bf16_mlp_matches_reference_at_bf16_tolerance(env):
    """BF16 variant (products on the tensor cores): forward output and
    gradients against the FP64 MLP; every product operand is rounded to
    bfloat16 (8-bit significand, relative spacing 2^-8), so the tolerance is a
    few times that spacing, against 1e-5 for FP32 (test above)."""
    torch, B = env
    rng = np.random.default_rng(3)
    widths = [64, 256, 256, 256, 128]
    m = B.dj_mlp_create(widths, seed=5)
    try:
        B.dj_mlp_set_precision(m, 1)
        p = B.dj_mlp_get_params(m).astype(np.float64)
        X = rng.normal(size=(128, 64))
        T = rng.normal(size=(128, 128))
        dX = torch.tensor(X, dtype=torch.float32, device="cuda")
        dT = torch.tensor(T, dtype=torch.float32, device="cuda")
        loss = B.dj_mlp_loss_grad(m, dX.data_ptr(), dT.data_ptr(), 0, 128)
        g = B.dj_mlp_get_grads(m).astype(np.float64)
        L_ref, g_ref = ref.loss_grad(p, widths, X, T, np.ones(128))
        dY = torch.empty((128, 128), device="cuda")
        B.dj_mlp_forward(m, dX.data_ptr(), 128, dY.data_ptr())
        Y_ref = ref.forward(p, widths, X)[-1]
        ey = np.abs(dY.cpu().numpy() - Y_ref).max() / np.abs(Y_ref).max()
        eg = np.abs(g - g_ref).max() / np.abs(g_ref).max()
        print(f"BF16 MLP: output rel err {ey:.2e}, gradient rel err {eg:.2e}, loss {loss:.4f} vs {L_ref:.4f}")
        assert abs(loss - L_ref) < 2e-2 * L_ref
        assert 1e-5 < ey < 3e-2 and eg < 5e-2  # rounded (not FP32), within BF16 accuracy
        B.dj_mlp_set_precision(m, 0)
        B.dj_mlp_forward(m, dX.data_ptr(), 128, dY.data_ptr())
        assert np.abs(dY.cpu().numpy() - Y_ref).max() < 1e-5 * np.abs(Y_ref).max()
    finally:
        B.dj_mlp_destroy(m)


@pytest.mark.parametrize("shape", [(200, 300, 150), (1, 64, 128), (256, 256, 256), (77, 40, 9)])
def test_tensor_core_products_match_cuda_core_bf16(env, shape):
    """The BF16 products on the tensor cores (tcgen05, precision 1) against the
    same BF16-rounded operands multiplied on the CUDA cores (precision 2): one
    linear layer (batch x in -> out; ragged sizes, a single row).  The forward
    product sees identical operands and agrees to FP32 accumulation-order
    rounding (2e-5); the weight gradient's operand dL/dY comes from that
    forward output, whose last-bit differences can move a value to the
    neighbouring bfloat16, so it agrees to a fraction of one BF16 spacing
    (1e-3 against 2^-8 = 3.9e-3)."""
    torch, B = env
    batch, n_in, n_out = shape
    rng = np.random.default_rng(11)
    X = rng.normal(size=(batch, n_in))
    T = rng.normal(size=(batch, n_out))
    dX = torch.tensor(X, dtype=torch.float32, device="cuda")
    dT = torch.tensor(T, dtype=torch.float32, device="cuda")
    out = {}
    for prec in (1, 2):
        m = B.dj_mlp_create([n_in, n_out], seed=2)
        try:
            B.dj_mlp_set_precision(m, prec)
            dY = torch.empty((batch, n_out), device="cuda")
            B.dj_mlp_forward(m, dX.data_ptr(), batch, dY.data_ptr())
            B.dj_mlp_loss_grad(m, dX.data_ptr(), dT.data_ptr(), 0, batch)
            out[prec] = (dY.cpu().numpy().astype(np.float64), B.dj_mlp_get_grads(m).astype(np.float64))
        finally:
            B.dj_mlp_destroy(m)
    (y1, g1), (y2, g2) = out[1], out[2]
    assert np.abs(y1 - y2).max() <= 2e-5 * np.abs(y2).max()
    assert np.abs(g1 - g2).max() <= 1e-3 * np.abs(g2).max()


@pytest.fixture(scope="module")
def coarse_ws(env):
    """A warm start trained by the library (dj_ws_train) on a coarse (6 mm)
    brain-sized ellipsoid: 2048 seeded loads of 1-4 mm relaxed from rest by the
    method itself (about 40 s), then the fit, whose held-out loads decide the
    polynomial order and whether the MLP is kept."""
    torch, B = env
    from paper_2106_14189_gb300.warmstart import WarmStart, load_cases
    p = W.ellipsoid_tet4(h=6e-3, seed=0, disp_range=(1e-3, 4e-3))
    ws = WarmStart(p, alpha=140.0, ramp_steps=750, tol=1e-5, epochs=1500, batch=128, mlp=-1)
    info = ws.train(load_cases(p, range(1000, 3048)))
    yield ws, info, p, load_cases(p, range(5000, 5016))
    ws.close()


def test_library_warm_start_relaxes_faster_than_rest(env, coarse_ws):
    """dj_ws_relax_to_tol on held-out loads: the fitted warm start reaches the
    same residual in fewer steps and less wall time (prediction and checks
    included) than relaxation from rest, and lands on the same equilibrium."""
    torch, B = env
    ws, info, p, T_test = coarse_ws
    # six patches, each displaced by one 3-vector: the targets span 18 dimensions
    assert info["n_kept"] >= 2000 and info["n_holdout"] == round(0.1 * info["n_kept"])
    assert 6 <= info["n_in_kept"] <= 18
    print("fit:", {k: info[k] for k in ("val_loss_first_order", "val_loss_second_order",
                                         "val_loss_polynomial_mlp", "quadratic_used", "mlp_used")})
    cold, warm = [], []
    with ws.mesh(T_test[0]) as m:
        ws.relax(T_test[0], "rest", m)  # warm-up: graph capture, first-use allocations
        ws.relax(T_test[0], "fitted", m)
        for t in T_test:
            rc = ws.relax(t, "rest", m)
            Uc = m.displacements()
            rw = ws.relax(t, "fitted", m)
            Uw = m.displacements()
            assert rc["status"] == 0 and rw["status"] == 0
            assert rc["residual"] <= 1e-5 and rw["residual"] <= 1e-5
            diff = np.abs(Uw - Uc).max() / np.abs(Uc).max()
            assert diff <= 1e-2, diff
            cold.append(rc)
            warm.append(rw)
    assert sum(r["fallback"] for r in warm) <= len(warm) // 4
    steps_c, steps_w = np.mean([r["steps"] for r in cold]), np.mean([r["steps"] for r in warm])
    ms_c, ms_w = np.mean([r["seconds"] for r in cold]) * 1e3, np.mean([r["seconds"] for r in warm]) * 1e3
    print(f"warm start: {steps_w:.0f} vs {steps_c:.0f} steps, {ms_w:.1f} vs {ms_c:.1f} ms")
    assert steps_w < 0.8 * steps_c and ms_w < ms_c


def test_library_warm_start_save_load_predicts_the_same(env, coarse_ws):
    torch, B = env
    ws, info, p, T_test = coarse_ws
    from paper_2106_14189_gb300.warmstart import WarmStart
    blob = ws.save()
    other = WarmStart(p)
    other.load(blob)
    for parts in (B.DJ_WS_PARTS_FITTED, B.DJ_WS_PARTS_POLYNOMIAL):
        a = ws.predict(T_test[1], parts).cpu().numpy()
        b = other.predict(T_test[1], parts).cpu().numpy()
        assert np.array_equal(a, b)
    assert other.info()["val_loss_polynomial"] == info["val_loss_polynomial"]
    other.close()
    with pytest.raises(B.DJError):
        B.dj_ws_load(blob[:-4])


def test_trained_network_gains_over_the_polynomial_part(env, coarse_ws):
    """What the trained MLP adds to the method without it: on the held-out
    training loads its map (polynomial part + MLP) has a lower loss than the
    polynomial part alone, so the fit keeps it; on 16 further held-out loads the
    relaxation from the full map reaches r <= 1e-5 in fewer steps and less wall
    time than from the polynomial part's prediction, which in turn beats
    relaxation from rest (the plain method)."""
    torch, B = env
    ws, info, p, T_test = coarse_ws
    assert info["mlp_used"] == 1 and info["quadratic_used"] == 1
    assert info["val_loss_polynomial_mlp"] < 0.5 * info["val_loss_polynomial"]
    arms = {a: [] for a in ("rest", "polynomial", "fitted")}
    with ws.mesh(T_test[0]) as m:
        for a in arms:
            ws.relax(T_test[0], a, m)  # warm-up
        for t in T_test:
            for a in arms:
                r = ws.relax(t, a, m)
                assert r["status"] == 0 and r["residual"] <= 1e-5
                arms[a].append(r)
    steps = {a: np.mean([r["steps"] for r in v]) for a, v in arms.items()}
    ms = {a: np.mean([r["seconds"] for r in v]) * 1e3 for a, v in arms.items()}
    print("held-out loss: polynomial %.2e, polynomial + MLP %.2e" %
          (info["val_loss_polynomial"], info["val_loss_polynomial_mlp"]))
    print("steps", {a: round(v) for a, v in steps.items()}, "ms", {a: round(v, 2) for a, v in ms.items()})
    assert sum(r["fallback"] for r in arms["fitted"]) == 0
    assert steps["fitted"] < 0.85 * steps["polynomial"] < 0.85 * steps["rest"]
    assert ms["fitted"] < ms["polynomial"] < ms["rest"]
