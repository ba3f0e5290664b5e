"""CPU oracle for the randomized orthogonal projection of Rokhlin & Tygert.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and
its Python binding) imports, links or executes anything here; only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it. It shares no code with the CUDA path: the only
module both sides use is ``workloads`` (seeded input generation, none of the
method's arithmetic).

Contents (all float64 unless stated):

* ``reference``    -- the plain definition: Householder QR of A^* and
                      Zb = b - Q(Q^* b), the row projection Q(Q^* b) and the
                      least-squares solution h = R^{-1} Q^* b (Eq. 1, Remark 4.1).
* ``paper_method`` -- the paper's algorithm step by step (Section 4): sketch
                      S = AG (Eq. 12), pivoted QR of S^* (Eq. 13), P^- (Eq. 15),
                      X column by column (steps a-e), Y = X^{-1} (Eq. 16), the
                      seven-step apply, and refinement (Remark 4.3).
* ``exact``        -- the exact projection of the stored float64 matrix, reached
                      by refinement (Remark 4.3) whose residuals are accumulated
                      in double-double arithmetic; the accuracy yardstick.
* ``philox``       -- Philox4x32-10 (Salmon et al., SC'11) and the maps from its
                      output to entries of the test matrix G.
* ``closed_form``  -- the exact projection for the paper's test family
                      (Eqs. 20-21), valid at any condition number.
* ``theory``       -- the probability bounds of Lemmas 2.1-2.3 (Eqs. 3-5) and
                      Observation 3.2 (Eq. 10).
* ``metrics``      -- the error measures of Section 5 (delta, epsilon) and
                      relative errors.
* ``gradient``     -- dL/dA and dL/dB of L = sum_j <g_j, Z b_j> (the adjoint of
                      Eq. 1) evaluated on the reference definition.

Parity pins: every function is checked in ``tests/test_oracle_*.py`` against
something other than itself (brute force in 60-digit arithmetic, the closed
form, invariants, library routines, values printed in the paper). The exact
pivot sequence of the pivoted QR on near-ties and the bitwise identity of the
Philox stream with other implementations of Philox are parity unpinned.
"""
from . import closed_form, exact, gradient, metrics, paper_method, philox, reference, theory  # noqa: F401
