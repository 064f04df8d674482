"""CPU oracle for the elastic Helmholtz shifted-Laplacian solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports this
package; it exists so that tests, the smoke check and the CPU baseline leg of
the benchmark can compare the CUDA path against a plain, slow, obviously
correct restatement of the paper (Treister & Yovel, "A hybrid shifted
Laplacian multigrid and domain decomposition preconditioner for the elastic
Helmholtz equations").

Everything is assembled as scipy.sparse complex128 matrices from Kronecker
products of 1D difference/averaging operators, in the order the paper states
the method (Sec. 2.1 discretization, Sec. 2.2 two-grid cycle and shift,
Sec. 2.3 multicolour DD, Sec. 3 mixed formulation and cell-wise relaxation,
Sec. 5 LFA).  The oracle shares no code with the CUDA path.

DOF ordering of the oracle (differs from the CUDA slot layout on purpose):
[u_1, ..., u_d, p]; u_k holds only the interior faces along direction k
((n_k - 1) values along k), p holds all cells; x is the fastest index.
"""
