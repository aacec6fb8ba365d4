"""FP64 CPU oracle for the heat-equation KKT system and its two-level time-DD preconditioner.

TEST INFRASTRUCTURE ONLY. This package is the slow, literal restatement of the method
of Cyr, "A 2-Level Domain Decomposition Preconditioner for KKT Systems with
Heat-Equation Constraints" (arXiv 2305.04421), used to check the CUDA path. Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it. The product path (``paper_2305_04421_gb300``) never imports it, and this
package never imports the product path. The two share no code: the only common
module is ``workloads`` (seeded input generators, no method arithmetic).

Modules
-------
problem   Section 2, Eqs 2-5: grid, 5-point Laplacian, J, L, the KKT matrix K, the RHS.
schwarz   Section 2 Eq 7 (block preconditioner, Pearson-Wathen S-hat) and Section 3
          Eqs 9-15 (RAS, RASQ, Nicolaides coarse space, two-level composition).
krylov    Section 4: right-preconditioned flexible GMRES (Saad), MGS orthogonalisation.
spectral  Exact per-mode direct solve of K (the DST diagonalises every spatial block):
          an independent pin of the final answer, not a step of the method.
mlp       NumPy forward/backward/Adam of the learned coarse correction's MLP (gradient pin).

All arithmetic is IEEE FP64. Every reading taken where the paper is silent, ambiguous or
garbled is stated, with its reason, at the function that takes it.
"""

from .problem import HeatKKT  # noqa: F401
