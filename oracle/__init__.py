"""FP64 reference implementations -- test infrastructure only.

Nothing in the product package imports this.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

* ``oracle.sim``   -- complex128 state-vector simulator in plain C (Eq. 1),
  gate matrices, fused-kernel unitaries.
* ``oracle.plan``  -- kernelization checks: plan validity (Theorem 2's
  topological equivalence), the analytic kernel cost of the paper's
  "Cost Function" section, brute-force optimal contiguous segmentation
  (Problem 1).
* ``oracle.mlp``   -- FP64 forward/backward/Adam for the learned cost model.
"""
