"""CPU oracle for the phi-function actions of exponential integrators.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, obviously-correct restatement of the paper
(Deka & Einkemmer, "A comparison of Leja- and Krylov-based iterative
schemes for Exponential Integrators", arXiv:2211.08948) in float64
NumPy/SciPy.  It shares no code with the CUDA library in
``paper_2211_08948_gb300/csrc``; the only module both sides use is
``synth`` (seeded input generators, no method arithmetic).

Modules
-------
phi          scalar phi_l(z) (Sec. 1 definition)
operators    2D periodic stencils: f(u) and J(u)w (Sec. 3: 2nd-order centred FD)
leja         Leja points, divided differences, power iteration, Newton
             interpolation of phi_l(hJ)v (Sec. 2.2), vertical form (Sec. 4)
kiops        KIOPS-style Krylov action on the augmented matrix (Sec. 2.1)
exact        exact references: FFT diagonalisation, dense expm of the
             augmented matrix (Theorem of Sec. 2.1)
integrators  the steps of Sec. 5: EXPRB43 (Eq. exprb43), EPIRK4s3 (Eq. epirk4s3),
             EPIRK4s3A (Eq. epirk4s3a), EXPRB53s3 (Eq. exprb5s3), EPIRK5P1 (its
             coefficient table), with Leja, KIOPS or LeKry (Sec. 5.1) and the
             vertical / horizontal grouping of Sec. 4
adaptive     traditional and cost step-size controllers (Sec. 2.3)
problems     the no-flow test problems of Sec. 3 (ADR, Allen-Cahn, Brusselator)
variants     finite-difference Jacobian actions (Sec. 4), augmented-matrix Leja
             (Appendix A)
mlp          MLP forward/backward/Adam for the learned spectral interval

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except where its docstring says
"parity unpinned".
"""
