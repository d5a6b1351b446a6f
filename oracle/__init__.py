"""FP64 CPU oracle of the i-DEQ inertial fixed-point iteration.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain, obviously-correct
restatement of the paper's method that the CUDA path is checked against.  Only the
test-suite, the package's ``smoke()`` self-check and the benchmark's CPU-baseline
leg may import it; the product path never calls it and must fail loudly when its
CUDA extension is missing.

Layout:
  operators.py  forward models A, adjoints, data term f and its derivatives
  nets.py       regulariser network N, g = 1/2 ||x - N(x)||^2, its gradient,
                Hessian-vector products and parameter gradients
  solver.py     the inertial iteration with restart and stopping (Alg. 1)
  adjoint.py    implicit differentiation of the fixed point (App. D.1.2)
  warmstart.py  the learned warm start x0 = A^T y + W(A^T y), MSE loss, Adam
All arithmetic is float64 NumPy; convolutions are explicit sums of shifted
matrix products, circular stencils explicit sums of np.roll.
"""
