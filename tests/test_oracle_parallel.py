"""The process-parallel driver of the oracle (oracle/parallel.py) reproduces
the serial oracle's trajectory up to FP64 rounding, for both formulations,
and the classical-TLED trajectory equals the DJ-TLED one (the paper's
equivalence, Sec. 5.1 and Fig. 4) to FP64 rounding."""
import numpy as np

from oracle import dynamics
from oracle.parallel import ParallelSolver
from paper_2106_14189_gb300 import workloads as W


def test_parallel_solver_matches_serial_oracle():
    p = W.cutout_cube(W.TET4, 6, W.TI, n_steps=60, extension=0.002)
    ref = dynamics.ExplicitSolver.from_problem(p).run(60)
    tl = dynamics.ExplicitSolver.from_problem(p, formulation="tled").run(60)
    with ParallelSolver(p, 3) as ps:
        U = ps.run(60)
    with ParallelSolver(p, 2, formulation="tled") as pt:
        Ut = pt.run(60)
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(U - ref).max() < 1e-11 * scale
    assert np.abs(Ut - tl).max() < 1e-11 * scale
    assert np.abs(tl - ref).max() < 1e-10 * scale
