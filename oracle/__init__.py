"""CPU oracle for DACP (dual application of Chebyshev polynomial, arXiv 2011.02107).

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or link
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. It shares no code with the CUDA path.

Plain, slow, float64 numpy code, written from the paper's equations in the
paper's order (Sec. II A-C, Appendices A-C) so that a reader can check it by
eye. Library primitives used as single steps: numpy fancy indexing, matrix
products and LAPACK ``eigh``/``eigvalsh``/``svd``.

Modules
  hamiltonian    matrix-free H.v (Sec. II intro, Sec. III) and the dense matrix,
                 with optional XX / YY pair couplings (XXZ, Heisenberg chains)
  chebyshev      T_k scalar definitions (Appendix A, Eqs. cheb, cheb2, rec)
  dacp           filter, evolution with directly recorded moments, assembly,
                 generalized eigensolve with rank removal (Sec. II, App. B-C)
  jordan_wigner  closed-form spectra: the h_z = 0 open Ising chain (Sec. III) and
                 the open XX chain in z-fields (free fermions)
  params         E_max upper bound (Lanczos) and DOS-based window (Sec. III)
  metrics        matching against an exact spectrum, local mean spacing
  mlp            plain forward/backward of the parameter MLP

Parity status: every function is pinned by a test in tests/test_oracle_*.py.
``params.kpm_window`` is a heuristic. It is pinned by its count identity and by
exact level counts of four N = 14 shards (dense eigh), to within 10 %; see the
module docstrings.
"""
