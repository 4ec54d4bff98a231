"""Learned warm start for dynamic relaxation: a thin owner of the library's
dj_ws object (include/dj_tled.h, csrc/warmstart.cu).

The library does all of it: the training data (the method's own relaxations
of seeded load cases, dj_ws_train, or caller-supplied fields through
dj_ws_fit), the POD bases and their scaling, the held-out choice of the
polynomial order and of the MLP, MLP training, prediction, and the
relaxation with its fallback rule (dj_ws_relax_to_tol).  This module only
builds the mesh from a workloads.Problem, marshals arguments and, for small
meshes, gathers training data with the batch API (many copies of the mesh
relaxed in one graph) before handing it to dj_ws_fit.  The paper names
learning methods only as future work (Sec. 8).
"""
from __future__ import annotations

import copy
from typing import List, Optional

import numpy as np

from . import binding as B
from . import workloads as W

ARMS = {"rest": B.DJ_WS_ARM_REST, "polynomial": B.DJ_WS_ARM_POLYNOMIAL, "fitted": B.DJ_WS_ARM_FITTED}


class WarmStart:
    """A warm start for one mesh (its nodes and prescribed DOFs).

    Mesh options (alpha, ramp_steps, check_every, precision) are those of the
    relaxations; ``ws_kw`` are dj_ws_params fields (n_in, n_out, hidden,
    epochs, batch, lr, lr_final, quadratic, mlp, mlp_input, mlp_bf16, holdout,
    seed, adaptive)."""

    def __init__(self, problem: W.Problem, tol: float = 1e-5, max_steps: int = 400000, alpha: float = 130.0,
                 ramp_steps: int = 400, check_every: int = 50, precision: int = 1, **ws_kw):
        self.p = problem
        self.tol, self.max_steps = tol, max_steps
        self.alpha, self.ramp_steps, self.check_every, self.precision = alpha, ramp_steps, check_every, precision
        self.params = B.ws_params(**ws_kw)
        self.ws = None
        self.n_dof = 3 * problem.n_nodes

    # ------------------------------------------------------------ problems --
    def problem_for(self, targets) -> W.Problem:
        q = copy.copy(self.p)
        q.bc_target = np.asarray(targets, dtype=np.float64)
        q.alpha, q.ramp_steps = self.alpha, self.ramp_steps
        return q

    def mesh_params(self):
        return dict(alpha=self.alpha, ramp_steps=self.ramp_steps, relax_check_every=self.check_every,
                    precision=self.precision)

    def mesh(self, targets=None) -> B.Mesh:
        return B.Mesh(self.problem_for(self.p.bc_target if targets is None else targets), **self.mesh_params())

    # ------------------------------------------------------------ training --
    def train(self, targets: np.ndarray, mesh: Optional[B.Mesh] = None) -> dict:
        """dj_ws_train: relax every load case from rest on the mesh, fit."""
        self.close()
        own = mesh is None
        if own:
            mesh = self.mesh(targets[0])
        try:
            self.ws = B.dj_ws_train(mesh.h, np.asarray(targets, dtype=np.float64), self.tol, self.max_steps,
                                    self.params)
        finally:
            if own:
                mesh.close()
        return self.info()

    def solve_batch(self, targets: List[np.ndarray], batch_size: int = 64):
        """Training data from the batch API (copies of a small mesh relaxed in
        one graph): (device tensor of the targets, device tensor of the relaxed
        fields, indices kept).  A batch that fails is redone case by case and
        failing cases are dropped."""
        import torch
        S = len(targets)
        Y = torch.empty((S, self.n_dof), dtype=torch.float32, device="cuda")
        kept = []
        for s0 in range(0, S, batch_size):
            chunk = targets[s0:s0 + batch_size]
            try:
                with B.Batch([self.problem_for(t) for t in chunk], **self.mesh_params()) as bt:
                    bt.relax(self.tol, self.max_steps)
                    for i in range(len(chunk)):
                        B.dj_batch_get_displacements_device(bt.b, i, Y[len(kept)].data_ptr())
                        kept.append(s0 + i)
                    bt.sync()
            except B.DJError:
                for i, t in enumerate(chunk):
                    with B.Mesh(self.problem_for(t), **self.mesh_params()) as m:
                        st, n, r = m.relax(self.tol, self.max_steps, raise_on_fail=False)
                        if st != 0:
                            continue
                        B.dj_get_displacements_device(m.h, Y[len(kept)].data_ptr())
                        m.sync()
                        kept.append(s0 + i)
        T = torch.tensor(np.asarray(targets, dtype=np.float32)[kept], device="cuda")
        return T, Y[:len(kept)].contiguous(), kept

    def fit(self, d_targets, d_fields, n_loads: int) -> dict:
        """dj_ws_fit on device tensors (n_loads x n_bc, n_loads x 3 n_nodes)."""
        self.close()
        self.ws = B.dj_ws_fit(self.p.bc_dof, self.p.n_nodes, d_targets.data_ptr(), d_fields.data_ptr(),
                              n_loads, self.params)
        return self.info()

    def info(self) -> dict:
        return B.dj_ws_get_info(self.ws)

    # ------------------------------------------------------------ solving ---
    def predict(self, targets, parts: int = B.DJ_WS_PARTS_FITTED):
        """Predicted nodal field (3 n_nodes floats on the device)."""
        import torch
        out = torch.empty(self.n_dof, dtype=torch.float32, device="cuda")
        B.dj_ws_predict(self.ws, targets, out.data_ptr(), parts)
        return out

    def relax(self, targets, arm: str, mesh: B.Mesh) -> dict:
        """dj_ws_relax_to_tol for one load case; `arm` is 'rest', 'polynomial'
        or 'fitted'.  Returns the result fields plus 'status'."""
        st, res = B.dj_ws_relax_to_tol(mesh.h, self.ws, targets, ARMS[arm], self.tol, self.max_steps,
                                       raise_on_fail=False)
        res["status"] = st
        return res

    def save(self) -> bytes:
        return B.dj_ws_save(self.ws)

    def load(self, blob: bytes):
        self.close()
        self.ws = B.dj_ws_load(blob)

    def close(self):
        if self.ws is not None:
            B.dj_ws_destroy(self.ws)
            self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def load_cases(problem: W.Problem, seeds) -> np.ndarray:
    return np.stack([W.ellipsoid_load_case(problem, int(s)) for s in seeds])
