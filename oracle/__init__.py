"""CPU FP64 oracle of the DiscoMatch dual / primal hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or execute anything in
this package. The product path (``paper_2310_08230_gb300``) never does, and the
two share no code: this package is written independently from the paper and
consumes only the raw seeded inputs of ``synth``.

Modules (each cites the passages it follows):
  problem.py  costs, candidates, product space, constraints of ILP (P), presolve
  bdd.py      constraint -> BDD compilation, BDD splitting (Alg. 3)
  mma.c       FP64 min-sum passes, min-marginals, deferred MMA half-passes
  solver.py   dual iteration driver, lower bounds (Eq. D)
  primal.py   min-marginal-driven rounding with propagation
  exact.py    exhaustive ILP optimum and LP relaxation of tiny instances

Every function is pinned by ``tests/test_oracle_*.py`` against values the paper
or the mathematics fix (Fig. BDD widths, brute-force min-marginals, closed
forms, weak duality, exhaustive optimum, invariants).
"""
