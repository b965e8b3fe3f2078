"""Plain FP64 CPU oracle for the Polya/SDP robust-stability method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It is a
slow, obviously-correct restatement of Kamyar, Peet & Peet, "Solving
Large-Scale Robust Stability Problems by Exploiting the Parallel Structure of
Polya's Theorem" (IEEE TAC 2013):

* ``polya``   -- monomial sets W_d, the index map, the beta and H coefficient
                 tables by the paper's recursions (Sec. III-A, Eqs. beta_init,
                 beta, H_init, H) and homogenisation (Sec. II).
* ``sdp``     -- the SDP elements C, B_i, a (Sec. III-B, Eqs. C, Cj, Ai, Aij, a)
                 both literally (every B_i materialised) and per block.
* ``ipm``     -- the primal-dual predictor-corrector interior-point method of
                 Sec. IV-A and Algorithm 2, with the Schur complement computed
                 from its definition (literal) or from the block formula.
* ``certify`` -- the stability certificate of Theorems 1 and 2.
* ``mlp``     -- the FP64 reference of the learned warm-start network (not in
                 the paper): a three-layer ReLU MLP, MSE loss and Adam.

Every floating-point computation is numpy float64.  The oracle shares no code
with the CUDA library; the only module both sides use is the seeded input
generator ``paper_1411_3769_gb300.synth``, which holds none of the method's
arithmetic.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against the paper's worked examples, closed forms, brute force and textbook
special cases; none is "parity unpinned" except the absolute iteration counts
of the IPM, which the paper does not print.
"""

from . import polya, sdp, ipm, certify  # noqa: F401
