"""CPU oracle for the Pauli-exponential state-vector path (test infrastructure).

Plain, slow, dense complex128 NumPy restatements of what the QForte paper
(arXiv:2108.04413) defines: the qubit basis of Eq. 3, the Pauli-string
exponential of Eq. 9 (with the factor -i*theta of the worked example Eq. 11-13),
exact operator averaging of the qubit Hamiltonian (Eq. 2, Eq. 18), the
Jordan-Wigner images of Eq. 15-16, the dUCC ansatz of Eq. 19, PQE's residuals
(Eq. 23-25) and quasi-Newton update (Eq. 26), ADAPT's operator gradients
(Eq. 21) and Trotterized evolution (Eq. 39).

This package is test infrastructure.  Only the test suite, the smoke check and
the CPU-baseline leg of the benchmark may import it.  The product path (the
CUDA library and its Python binding) never imports or calls it, and it shares
no code with that path: the only common module is `workloads`, which draws the
seeded random inputs and holds none of the method's arithmetic.

Every function is pinned by the `-m "not gpu"` tests against closed forms,
textbook routines (scipy.linalg.expm, Kronecker-product matrices, numpy.linalg
eigenvalues) or values printed in the paper (Tab. 1).
"""
