"""FP64 CPU oracle for the DJ-TLED time step (arXiv 2106.14189).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may use it.  It shares no code with the CUDA library
(``paper_2106_14189_gb300/csrc``); the only common module is the seeded input
generator ``paper_2106_14189_gb300.workloads``, which holds none of the
method's arithmetic.

Modules
-------
elements   natural-coordinate shape-function derivatives H_xi (Eq. 6, Sec. 7 on
           volume coordinates), reference Jacobian 0J (Eq. 3), element volume.
djtled     paper-literal DJ-TLED: G matrices (App. B), m-vectors and M2
           (App. C), I_im tensors (Table 2), invariants (Table 1) and nodal
           forces (Table 3, Algorithm 1).
tled       classical TLED written independently from the textbook: deformation
           gradient, right Cauchy-Green tensor, second Piola-Kirchhoff stress
           and F = X S 0B 0V (Eq. 4, Eq. 54-55, Table 8).  Used to pin djtled.
hourglass  displacement-based hourglass control for 1-point H8 (the paper only
           cites its source; reading documented in the module).
dynamics   lumped mass, critical time step (Eq. 14), assembly, central
           difference with mass-proportional damping (Eq. 13), prescribed
           displacements, residual and dynamic relaxation.
mlp        FP64 multilayer perceptron forward/backward and Adam for the learned
           warm start, plus the POD basis.

Every function is written for clarity, not speed: vectorised over elements with
numpy, no blocking or fusion beyond what the cited formula states.
"""
