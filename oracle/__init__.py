"""Oracle: a plain, slow, FP64 CPU statement of what the Birkhoff hot path computes.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import or run it. The product path (the
CUDA library and its Python binding in ``paper_2509_01855_gb300``) never imports it and shares
no code, table or constant generator with it.

Every function cites the passage of arXiv 2509.01855 ("A Million-Point Fast Trajectory
Optimization Solver") that it restates. Where the paper is silent or misprinted, the reading
taken is stated in the docstring.

Modules
-------
grid      CGL nodes (Eq. CGLpts), Lagrange basis, Clenshaw-Curtis weights.
birkhoff  dense B^a from its definition (Eqs. xN=Birka+b, birk-conditions, manyDefs), the
          FastBV chain (Fastv2a, Eq. c_k=bydef, Eq. chatk=, Fasta2v), closed-form integrals
          of T_k (Eq. intChebPoly=), B-tilde, FastBccV and the corrected FastPinvY sweep.
problems  dynamics f, its Jacobians and Hessians for the problem kinds of the library.
kkt       dense KKT of the a-form discretisation (Eq. Prob-PNa) and a Newton-Lagrange driver.
"""
