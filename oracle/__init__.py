"""FP64 CPU oracle for the H^2-ULV factorization and substitution.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links
this package. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

It is a plain, slow, step-by-step restatement of the method of Ma & Yokota,
"An inherently parallel H^2-ULV factorization for solving dense linear systems
on GPUs" (arXiv 2502.02395):

  kernels.py    the kernel functions (Eq. 35, Eq. 36 and the variants the
                workloads use)
  tree.py       the binary cluster tree, admissibility and near/far lists
                (Section 3.3, Section 6.2, Section 6.3)
  construct.py  the H^2 construction with the pre-factorization basis
                (Algorithm 1, Eq. 22-23, Section 3.5)
  ulv.py        complement bases (Eq. 6-7), the level-by-level ULV
                factorization (Algorithm 2 / Algorithm 4, with partial-pivot
                LU for the redundant blocks), the naive substitution
                (Algorithm 3) and the parallel substitution (Eq. 24-31), the
                H^2 matrix-vector product and iterative refinement
  dense.py      dense assembly and a textbook partial-pivot LU solve
  mlp.py        the rank predictor's 16-64-64-1 network (forward, loss and
                chain-rule gradient), the spec extension that learns
                the ranks Algorithm 1's compression keeps
  instance.py   writes an H^2 instance to a .npz file for the library's
                h2_import

Every floating-point step is FP64. Library primitives (matmul, QR with column
pivoting, LU) serve as steps; there is no blocking or reordering beyond what
the algorithms state.

Parity status of each part is listed in ``PARITY`` below. The construction's
sampling rule and admissibility constant are choices the paper leaves open;
they are fixed here and checked only through the residual ("parity unpinned").
"""

PARITY = {
    "kernels": "pinned: closed forms at fixed points (tests/test_oracle_pins.py)",
    "tree": "pinned: partition invariants and brute-force admissibility",
    "construct.sampling_rule": "parity unpinned (the paper does not fix it)",
    "construct.prefactor": "pinned: dropped Eq. 21 fill-ins fall with tol only with the close-field term; "
                           "that term scales with the inverse diagonal (tests/test_oracle_pins.py)",
    "construct.id": "pinned: exact-rank kernel gives an exact ID; interpolation rows",
    "ulv.complement_basis": "pinned: orthogonality <= 1e-13, span of X",
    "ulv.factor": "pinned: exact-rank kernel equals dense LU to ~1e-12; brute force on tiny trees",
    "ulv.solve_parallel": "pinned: equals the naive Algorithm 3 on the exact-rank kernel",
    "ulv.matvec": "pinned: equals the dense assembly of the H^2 matrix",
    "ulv.refine": "pinned: residual reaches the target; matches dense solve within the H^2 error",
    "mlp": "pinned: central finite differences of the loss; closed form for a constant network",
    "dense": "pinned: numpy.linalg.solve on random systems",
}
