"""FP64 CPU oracle for the graph neural preconditioner and FGMRES.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import anything from this package.  The
product path (``paper_2406_00809_gb300`` and its CUDA library) never imports it and
shares no code, table or helper with it; the only common dependency is the seeded
problem generator ``paper_2406_00809_gb300.inputs``, which holds none of the method's
arithmetic.

Modules
-------
gnp_ref      gamma normalisation (Eq. 6), scaling s (Eq. 8), MLP encoder/decoder
             (Sec. 2.3 item 3, Sec. 3 "Hyperparameters"), Res-GCONV (Eq. 7) and the
             residual variant H + ReLU(A_hat H W); hand-derived backward; l1 residual
             loss (Sec. 3); Adam (Kingma & Ba).
krylov_ref   FGMRES with a nonlinear M (Algorithm 1, Eq. 1) with MGS or CGS2
             orthogonalisation and Givens least squares; a separate textbook GMRES for
             pinning; the Arnoldi process (Eq. 4) and the training-pair sampler (Eq. 5).
precond_ref  the Jacobi and inner-GMRES preconditioners the paper compares with
             (Sec. 3 "Compared methods").
metrics_ref  the Iter-AUC and Time-AUC convergence metrics (Sec. 3 "Evaluation
             metrics").
philox_ref   Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the
             Box-Muller transform, used for the random draws of training.

Everything is float64 unless a function says otherwise.
"""
