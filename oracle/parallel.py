"""Process-parallel driver of the FP64 oracle (test infrastructure, like the
rest of this package): the oracle's explicit solver (dynamics.ExplicitSolver)
with its internal-force sum split over host processes, one contiguous block
of elements each.  Every process evaluates the oracle's own element forces of
its block and assembles them over all nodes in ascending element id
(dynamics.Model.internal_forces); the driver adds the block sums in block
order.  The result is the serial oracle's up to the FP64 rounding of that
regrouped sum (checked in tests/test_oracle_parallel.py); nothing here changes
the method's arithmetic.  Processes are started with the spawn method, so the
driver may be created after CUDA was initialised in the calling process.
"""
import copy

import numpy as np

from . import dynamics

PER_ELEMENT = ("conn", "model", "mu", "kappa", "rho", "eta_a", "eta_b", "c01", "a_dir", "b_dir")


def _block_worker(conn, problem, e0, e1, formulation):
    sub = copy.copy(problem)
    for k in PER_ELEMENT:
        v = getattr(problem, k)
        if v is not None:
            setattr(sub, k, np.asarray(v)[e0:e1])
    m = dynamics.Model.from_problem(sub, formulation=formulation)
    conn.send(True)
    while True:
        U = conn.recv()
        if U is None:
            break
        conn.send(m.internal_forces(U))


class ParallelSolver:
    """dynamics.ExplicitSolver of `problem` whose internal forces are summed
    over n_proc spawned processes.  Use as a context manager or call close()."""

    def __init__(self, problem, n_proc, formulation="djtled", dt=None):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.solver = dynamics.ExplicitSolver.from_problem(problem, dt=dt, formulation=formulation)
        E = problem.n_elems
        n_proc = max(1, min(int(n_proc), E))
        cuts = np.linspace(0, E, n_proc + 1).astype(int)
        self.pipes, self.procs = [], []
        for i in range(n_proc):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_block_worker, args=(b, problem, int(cuts[i]), int(cuts[i + 1]), formulation),
                             daemon=True)
            pr.start()
            self.pipes.append(a)
            self.procs.append(pr)
        for a in self.pipes:
            a.recv()
        self.solver.m.internal_forces = self._forces

    def _forces(self, U):
        for a in self.pipes:
            a.send(U)
        F = self.pipes[0].recv()
        for a in self.pipes[1:]:
            F = F + a.recv()
        return F

    @property
    def U(self):
        return self.solver.U

    @property
    def dt(self):
        return self.solver.dt

    def step(self):
        self.solver.step()

    def run(self, n_steps):
        return self.solver.run(n_steps)

    def close(self):
        for a in self.pipes:
            try:
                a.send(None)
            except Exception:
                pass
        for pr in self.procs:
            pr.join(timeout=10)
            if pr.is_alive():
                pr.terminate()
        self.pipes, self.procs = [], []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
