"""CPU oracle for camera covariance propagation (TEST INFRASTRUCTURE ONLY).

A plain, slow, FP64 CPU restatement of the method of Polic, Foerstner and
Pajdla, "Fast and Accurate Camera Covariance Computation for Large 3D
Reconstruction" (Sec. 3 problem formulation, Sec. 4 solution method).  It
exists to check the CUDA path and shares no code with it.  Only the test suite,
`__graft_entry__.smoke()` and the `cpu_baseline` / reference leg of `bench.py`
may import it; the library itself never does.

Modules
  camera       projection model and forward-mode (dual number) Jacobians
  information  blocks of the Fisher information M = J^T Sigma_u^-1 J (Eq. normal equations)
  nullspace    the similarity-gauge nullspace H, paper route J_r H_r = B (Sec. 4.1)
  covariance   conditioned, permuted bordered system, Schur complement Z_p,
               LU inverse and camera blocks Sigma_P = S_P Z_s S_P (Sec. 4.2)
  brute        extended-precision ground truth for tiny scenes (Sec. 6: SVD of
               M with exactly seven zero singular values; bordered inverse)
  metrics      per-block error measures, including the paper's err (Sec. 6)
  surrogate    the learned per-camera covariance predictor (not in the paper):
               features, targets, bf16-rounding MLP forward/backward, Adam

Parity status: every function here is pinned by a `-m "not gpu"` test against
something other than itself (closed forms, complex-step derivatives, dense
brute force in 40-digit arithmetic, invariants); the paper prints no worked
numerical example, so no pin uses printed values.
"""
