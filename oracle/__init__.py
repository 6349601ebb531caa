"""CPU oracle for the LDG multigrid hot path (arXiv 2412.12506, Saye).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
the paper's method, written to check the CUDA library against.  Only the test
suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference
leg may import it.  The product path (the C-ABI library and its Python
binding) never imports, links or calls anything here, and this package never
imports the product.  The two share no code; only the seeded input generator
(``paper_2412_12506_gb300.inputs``, which holds no method arithmetic) feeds
both.

Modules
  ldg        Sec. 2.1: tensor-product Legendre basis, discrete gradient G_a with
             viscosity-upwinded one-sided fluxes, mu-weighted mass M_mu,
             penalty E, and A = sum_a G_a^T M_mu G_a + E.
  multigrid  Sec. 2.2-2.3: injection I, operator coarsening, block Jacobi
             (Eq. Jsmooth), balanced block SAI (Sec. 2.3.3, Eqs. B1/BT),
             bottom pseudo-inverse, V-cycle (Algorithm 1).
  krylov     Sec. 2.2 / 2.4: preconditioned CG, eta (Eq. eta).

Parity status: every function is pinned by a test in tests/test_oracle_*.py
against a closed form, an invariant, a brute-force computation or a value
printed in the paper (Table tab:sizes), except the items listed as
"parity unpinned" in the module headers.
"""
