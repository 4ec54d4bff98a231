"""Learned warm start for dynamic relaxation.

A small MLP maps the prescribed surface displacements of a load case to an
initial nodal field for dynamic relaxation (the paper names learning methods
only as future work, Sec. 8).  Everything numerical runs in the CUDA library:

* training data: the method's own relaxed solutions, computed in batches of
  load cases on copies of the mesh (dj_batch_relax_to_tol);
* inputs: the leading POD coefficients of the prescribed-displacement vector,
  outputs: the leading POD coefficients of the relaxed field (dj_pod_fit /
  dj_pod_project / dj_pod_expand);
* the map from input to output coefficients: a ridge least-squares polynomial
  part on the kept input coefficients and their pairwise products
  (dj_quad_features, dj_linear_fit / dj_linear_apply) plus an MLP trained on
  what it leaves (dj_mlp_loss_grad / dj_mlp_adam_step / dj_mlp_forward), kept
  only when it improves the held-out error.

A relaxation from the predicted field uses plain DJ-TLED relaxation both as
fallback and as arbiter: if the predicted field inverts an element or has a
larger residual than the prescribed-values-only field, the solve restarts from
rest; the result is always a relaxation of the method to the same tolerance.
Torch provides device buffers and a few one-time tensor operations of the
set-up (scaling of the POD bases by the coefficient spread).
"""
from __future__ import annotations

import copy
import time
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import binding as B
from . import workloads as W


@dataclass
class RelaxResult:
    steps: int
    residual: float
    seconds: float
    warm: bool
    fallback: bool
    status: int
    predict_seconds: float = 0.0


class WarmStart:
    def __init__(self, problem: W.Problem, n_in: int = 64, n_out: int = 128,
                 hidden=(256, 256, 256), seed: int = 0, alpha: float = 130.0,
                 ramp_steps: int = 400, check_every: int = 50, tol: float = 1e-5,
                 max_steps: int = 400000, precision: int = 1, linear: bool = True,
                 quadratic: bool = True, adaptive: bool = False):
        import torch
        self.torch = torch
        self.p = problem
        self.n_in, self.n_out = n_in, n_out
        self.widths = [n_in, *hidden, n_out]
        self.seed = seed
        self.alpha, self.ramp_steps, self.check_every = alpha, ramp_steps, check_every
        self.tol, self.max_steps, self.precision = tol, max_steps, precision
        self.adaptive = adaptive  # relax with dj_relax_adaptive (damping estimated on the way)
        self.linear, self.quadratic = linear, quadratic
        self.quadratic_allowed = quadratic
        self.n_bc = problem.bc_dof.size
        self.n_dof = 3 * problem.n_nodes
        self.mlp = None
        self.use_mlp = True
        self.dev = torch.device("cuda")
        self.bc_index = torch.as_tensor(problem.bc_dof, device=self.dev)
        self.buf_c = torch.empty((1, n_in), device=self.dev)
        self.buf_q = torch.empty((1, n_out), device=self.dev)
        self.buf_field = torch.empty(self.n_dof, device=self.dev)
        self.buf_rest = torch.zeros(self.n_dof, device=self.dev)

    # ------------------------------------------------------------ problems --
    def problem_for(self, targets) -> W.Problem:
        q = copy.copy(self.p)
        q.bc_target = np.asarray(targets, dtype=np.float64)
        q.alpha, q.ramp_steps = self.alpha, self.ramp_steps
        return q

    def mesh_params(self):
        return dict(alpha=self.alpha, ramp_steps=self.ramp_steps,
                    relax_check_every=self.check_every, precision=self.precision)

    # --------------------------------------------------------------- data ---
    def solve_batch(self, targets: List[np.ndarray], batch_size: int = 64):
        """Relax every load case from rest.  Returns (S' x n_dof) device tensor of
        relaxed fields (one row per snapshot), the indices of the load cases that
        were kept, and the step counts.  A batch whose relaxation fails (an
        element inverts) is redone case by case and the failing cases are
        dropped."""
        torch = self.torch
        S = len(targets)
        Y = torch.empty((S, self.n_dof), dtype=torch.float32, device=self.dev)
        steps, kept = [], []
        for s0 in range(0, S, batch_size):
            chunk = targets[s0:s0 + batch_size]
            try:
                with B.Batch([self.problem_for(t) for t in chunk], **self.mesh_params()) as bt:
                    st, n, r = bt.relax(self.tol, self.max_steps)
                    for i in range(len(chunk)):
                        B.dj_batch_get_displacements_device(bt.b, i, Y[len(kept)].data_ptr())
                        kept.append(s0 + i)
                    bt.sync()
                    steps.append(n)
            except B.DJError:
                for i, t in enumerate(chunk):
                    with B.Mesh(self.problem_for(t), **self.mesh_params()) as m:
                        st, n, r = m.relax(self.tol, self.max_steps, raise_on_fail=False)
                        if st != 0:
                            continue
                        B.dj_get_displacements_device(m.h, Y[len(kept)].data_ptr())
                        m.sync()
                        kept.append(s0 + i)
                        steps.append(n)
        return Y[:len(kept)], kept, steps

    def solve_sequential(self, targets: List[np.ndarray]):
        """As solve_batch, one load case after the other on a single mesh (large
        meshes, where building a batch of copies costs more than it saves)."""
        torch = self.torch
        S = len(targets)
        Y = torch.empty((S, self.n_dof), dtype=torch.float32, device=self.dev)
        steps, kept = [], []
        zeros = np.zeros((self.p.n_nodes, 3))
        with B.Mesh(self.problem_for(targets[0]), **self.mesh_params()) as m:
            for i, t in enumerate(targets):
                B.dj_mesh_update_bc_targets(m.h, t)
                m.set_displacements(zeros)
                B.dj_set_step(m.h, 0)
                st, n, r = self._relax(m)
                if st != 0:
                    continue
                B.dj_get_displacements_device(m.h, Y[len(kept)].data_ptr())
                kept.append(i)
                steps.append(n)
            m.sync()
        return Y[:len(kept)], kept, steps

    # ---------------------------------------------------------------- fit ---
    def fit(self, T_host: np.ndarray, Y: "torch.Tensor", epochs: int = 400, batch: int = 256,
            lr: float = 1e-3, lr_final: float = 1e-5):
        """T_host: (S x n_bc) load targets, Y: (S x n_dof) device relaxed fields."""
        torch = self.torch
        S = T_host.shape[0]
        dT = torch.tensor(np.asarray(T_host, dtype=np.float32), device=self.dev)  # rows = snapshots
        self.mean_in = torch.empty(self.n_bc, device=self.dev)
        self.modes_in = torch.empty((self.n_bc, self.n_in), device=self.dev)
        self.mean_out = torch.empty(self.n_dof, device=self.dev)
        self.modes_out = torch.empty((self.n_dof, self.n_out), device=self.dev)
        self.sig_in = B.dj_pod_fit(dT.data_ptr(), self.n_bc, S, self.n_in, self.mean_in.data_ptr(),
                                   self.modes_in.data_ptr())
        self.sig_out = B.dj_pod_fit(Y.data_ptr(), self.n_dof, S, self.n_out, self.mean_out.data_ptr(),
                                    self.modes_out.data_ptr())
        # scale the bases so that coefficients have unit spread over the training set;
        # modes beyond the numerical rank of the snapshots (a load family of low
        # dimension has few input modes) are switched off instead of being
        # scaled up to unit-variance noise
        def spreads(sig, rel):
            keep = sig > rel * max(sig[0], 1e-300)
            return np.where(keep, sig / np.sqrt(S), 0.0), keep
        # (the Gram matrix of dj_pod_fit is stored in FP32, so singular values
        # below ~3e-4 sigma_1 are rounding: the input threshold sits above that)
        s_in_np, self.keep_in = spreads(self.sig_in, 1e-3)
        s_out_np, self.keep_out = spreads(self.sig_out, 1e-6)
        inv_in = np.where(self.keep_in, 1.0 / np.where(self.keep_in, s_in_np, 1.0), 0.0)
        self.modes_in *= torch.tensor(inv_in, dtype=torch.float32, device=self.dev)
        s_out = torch.tensor(s_out_np, dtype=torch.float32, device=self.dev)
        self.modes_out *= s_out
        Xc = torch.empty((S, self.n_in), device=self.dev)
        Qc = torch.empty((S, self.n_out), device=self.dev)
        B.dj_pod_project(self.modes_in.data_ptr(), self.mean_in.data_ptr(), self.n_bc, self.n_in,
                         dT.data_ptr(), S, Xc.data_ptr())
        # outputs: coefficients in the scaled output basis (modes_out has spread s_out^2)
        inv_out2 = np.where(self.keep_out, 1.0 / np.where(self.keep_out, s_out_np, 1.0) ** 2, 0.0)
        proj = self.modes_out * torch.tensor(inv_out2, dtype=torch.float32, device=self.dev)
        self.proj_out = proj
        B.dj_pod_project(proj.data_ptr(), self.mean_out.data_ptr(), self.n_dof, self.n_out,
                         Y.data_ptr(), S, Qc.data_ptr())
        # a seeded tenth of the snapshots is held out to decide whether the MLP
        # improves on the linear part alone
        rng = np.random.default_rng(self.seed)
        perm = rng.permutation(S)
        n_val = max(1, S // 10) if S >= 20 else 0
        val_idx = torch.tensor(perm[:n_val], device=self.dev)
        tr_idx = torch.tensor(perm[n_val:], device=self.dev)
        Xv, Qv = Xc.index_select(0, val_idx).contiguous(), Qc.index_select(0, val_idx).contiguous()
        Xc, Qc = Xc.index_select(0, tr_idx).contiguous(), Qc.index_select(0, tr_idx).contiguous()
        S = S - n_val
        # polynomial part of the map by ridge least squares on the kept input
        # coefficients and (quadratic) their pairwise products; the MLP learns
        # the rest
        # loss weights: output variance shares, so the loss tracks the field error
        var = np.where(self.keep_out, self.sig_out ** 2, 0.0)
        self.w = torch.tensor(var / var.mean(), dtype=torch.float32, device=self.dev)

        def fit_poly(quadratic):
            """ridge fit of the polynomial part; (W, features, held-out loss)"""
            self.quadratic = quadratic
            n_k = int(self.keep_in.sum())
            self.n_feat = n_k + (n_k * (n_k + 1) // 2 if quadratic else 0)
            W = torch.zeros((self.n_out, self.n_feat), device=self.dev)
            F = self._features(Xc, S)
            B.dj_linear_fit(F.data_ptr(), Qc.data_ptr(), S, self.n_feat, self.n_out,
                            1e-4 if quadratic else 1e-6, W.data_ptr())
            loss = None
            if n_val:
                Fv = self._features(Xv, n_val)
                pv = torch.zeros((n_val, self.n_out), device=self.dev)
                B.dj_linear_apply(W.data_ptr(), self.n_out, self.n_feat, Fv.data_ptr(), n_val, 1.0, 0.0,
                                  pv.data_ptr())
                loss = float(((pv - Qv) ** 2 * self.w).mean())
            return W, F, loss

        # polynomial part of the map by ridge least squares on the kept input
        # coefficients and, if it does better on the held-out snapshots, their
        # pairwise products; the MLP learns the rest
        want_quadratic = self.quadratic_allowed
        self.val_loss_first_order = self.val_loss_second_order = None
        if self.linear:
            W, Ftr, l1 = fit_poly(False)
            self.val_loss_first_order = l1
            n_k = int(self.keep_in.sum())
            if want_quadratic and S > 2 * n_k and n_k + n_k * (n_k + 1) // 2 <= 1024:
                W2, F2, l2 = fit_poly(True)
                self.val_loss_second_order = l2
                if l1 is None or (l2 is not None and l2 < l1):
                    W, Ftr = W2, F2
                else:
                    fit_poly(False)
            self.W_lin = W
            B.dj_linear_apply(self.W_lin.data_ptr(), self.n_out, self.n_feat, Ftr.data_ptr(), S, -1.0, 1.0,
                              Qc.data_ptr())
        else:
            self.quadratic = False
            self.n_feat = int(self.keep_in.sum())
            self.W_lin = torch.zeros((self.n_out, self.n_feat), device=self.dev)
        self.buf_f = torch.empty((1, self.n_feat), device=self.dev)
        Fv = self._features(Xv, n_val) if n_val else None
        if self.mlp is not None:
            B.dj_mlp_destroy(self.mlp)
        self.mlp = B.dj_mlp_create(self.widths, seed=self.seed)
        n_iter = epochs * max(1, S // batch)
        losses = []
        bsz = min(batch, S)
        for it in range(n_iter):
            idx = torch.tensor(rng.choice(S, size=bsz, replace=False), device=self.dev)
            xb = Xc.index_select(0, idx).contiguous()
            tb = Qc.index_select(0, idx).contiguous()
            want = (it % 200 == 0) or it == n_iter - 1
            loss = B.dj_mlp_loss_grad(self.mlp, xb.data_ptr(), tb.data_ptr(), self.w.data_ptr(), bsz,
                                      want_loss=want)
            if want:
                losses.append((it, loss))
            frac = it / max(1, n_iter - 1)
            B.dj_mlp_adam_step(self.mlp, lr * (lr_final / lr) ** frac)
        torch.cuda.synchronize()
        self.losses = losses
        # validation: weighted error of the output coefficients, linear part
        # alone against linear part + MLP; the MLP is kept only if it helps
        self.use_mlp = True
        self.val_loss_linear = self.val_loss = None
        if n_val > 0:
            lin = torch.zeros((n_val, self.n_out), device=self.dev)
            B.dj_linear_apply(self.W_lin.data_ptr(), self.n_out, self.n_feat, Fv.data_ptr(), n_val, 1.0, 0.0,
                              lin.data_ptr())
            full = torch.empty((n_val, self.n_out), device=self.dev)
            B.dj_mlp_forward(self.mlp, Xv.data_ptr(), n_val, full.data_ptr())
            full += lin
            self.val_loss_linear = float(((lin - Qv) ** 2 * self.w).mean())
            self.val_loss = float(((full - Qv) ** 2 * self.w).mean())
            self.use_mlp = self.val_loss < self.val_loss_linear
        return losses

    # ------------------------------------------------------------ predict ---
    def predict(self, targets: np.ndarray) -> "torch.Tensor":
        """Predicted nodal field (n_dof floats on the device) for one load case."""
        torch = self.torch
        t = torch.as_tensor(np.asarray(targets, dtype=np.float32)).to(self.dev, non_blocking=True)
        c, q, out = self.buf_c, self.buf_q, self.buf_field
        B.dj_pod_project(self.modes_in.data_ptr(), self.mean_in.data_ptr(), self.n_bc, self.n_in,
                         t.data_ptr(), 1, c.data_ptr())
        if self.use_mlp:
            B.dj_mlp_forward(self.mlp, c.data_ptr(), 1, q.data_ptr())
        f = self._features(c, 1, out=self.buf_f)
        B.dj_linear_apply(self.W_lin.data_ptr(), self.n_out, self.n_feat, f.data_ptr(), 1, 1.0,
                          1.0 if self.use_mlp else 0.0, q.data_ptr())
        B.dj_pod_expand(self.modes_out.data_ptr(), self.mean_out.data_ptr(), self.n_dof, self.n_out,
                        q.data_ptr(), 1, out.data_ptr())
        return out

    def _features(self, X: "torch.Tensor", rows: int, out=None) -> "torch.Tensor":
        """Inputs of the polynomial part: the kept (leading) input coefficients
        and, with quadratic=True, their pairwise products (dj_quad_features)."""
        torch = self.torch
        n_k = int(self.keep_in.sum())
        if out is None:
            out = torch.empty((rows, self.n_feat), device=self.dev)
        if self.quadratic:
            B.dj_quad_features(X.data_ptr(), rows, self.n_in, n_k, out.data_ptr())
        else:
            out.copy_(X[:, :n_k])
        return out

    def reconstruct(self, field: "torch.Tensor") -> "torch.Tensor":
        """Projection of a nodal field (n_dof floats on the device) onto the
        output basis and back: the best the output representation can do."""
        torch = self.torch
        q = torch.empty((1, self.n_out), device=self.dev)
        out = torch.empty(self.n_dof, device=self.dev)
        B.dj_pod_project(self.proj_out.data_ptr(), self.mean_out.data_ptr(), self.n_dof, self.n_out,
                         field.data_ptr(), 1, q.data_ptr())
        B.dj_pod_expand(self.modes_out.data_ptr(), self.mean_out.data_ptr(), self.n_dof, self.n_out,
                        q.data_ptr(), 1, out.data_ptr())
        return out

    # -------------------------------------------------------------- solve ---
    def relax(self, targets: np.ndarray, warm: bool, mesh: Optional[B.Mesh] = None) -> RelaxResult:
        """Relax one load case from rest (warm=False) or from the prediction."""
        torch = self.torch
        own = mesh is None
        if own:
            mesh = B.Mesh(self.problem_for(targets), **self.mesh_params())
        else:
            B.dj_mesh_update_bc_targets(mesh.h, targets)
            mesh.set_displacements(np.zeros((self.p.n_nodes, 3)))
            B.dj_set_step(mesh.h, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fallback = False
        if warm:
            field = self.predict(targets)
            r_warm, inverted = B.dj_evaluate_field(mesh.h, field.data_ptr())
            bc_only = self.buf_rest
            bc_only[self.bc_index] = torch.as_tensor(np.asarray(targets, dtype=np.float32)).to(self.dev)
            r_rest, _ = B.dj_evaluate_field(mesh.h, bc_only.data_ptr())
            if inverted or not (r_warm < r_rest):
                fallback = True
            else:
                B.dj_set_displacements_device(mesh.h, field.data_ptr())
                B.dj_set_step(mesh.h, self.ramp_steps)
        t_pred = 0.0
        if warm:
            torch.cuda.synchronize()
            t_pred = time.perf_counter() - t0
        st, n, r = self._relax(mesh)
        if warm and not fallback and st != 0:
            # the relaxation from the prediction failed (an element inverted on
            # the way): the same solve from rest decides
            fallback = True
            mesh.set_displacements(np.zeros((self.p.n_nodes, 3)))
            B.dj_set_step(mesh.h, 0)
            st, n2, r = self._relax(mesh)
            n += n2
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        if own:
            mesh.close()
        return RelaxResult(steps=n, residual=r, seconds=sec, warm=warm and not fallback,
                           fallback=fallback, status=st, predict_seconds=t_pred)

    def _relax(self, mesh):
        if self.adaptive:
            st, n, r, _ = mesh.relax_adaptive(self.tol, self.max_steps, raise_on_fail=False)
            return st, n, r
        return mesh.relax(self.tol, self.max_steps, raise_on_fail=False)

    def close(self):
        if self.mlp is not None:
            B.dj_mlp_destroy(self.mlp)
            self.mlp = None


def load_cases(problem: W.Problem, seeds) -> np.ndarray:
    return np.stack([W.ellipsoid_load_case(problem, int(s)) for s in seeds])
