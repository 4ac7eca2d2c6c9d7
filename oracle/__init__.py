"""Plain FP64 CPU oracle for the batched node-bound engine.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, header, table or helper with the CUDA library in
``paper_2605_22188_gb300/``; both sides only consume the same seeded inputs
produced by ``paper_2605_22188_gb300.synth`` (which holds none of the method's
arithmetic).

The oracle follows Liu & Lodi, "From Sequential Nodes to GPU Batches:
Parallel Branch and Bound for Optimal k-Sparse GLMs":

* ``losses``  -- the separable GLM losses, their derivatives and conjugates
  (§4.2 separable form, §4.4 Eq. (batched_dual_value_component)) and the Huber
  function H_M named in §3 Eq. (prelim_node_conjugate).
* ``node``    -- one BnB node: the proximal step of §3 Eq.
  (pgd_step_vector_form) with prox of rho*g* by Algorithm 1 (App. B), the
  primal term g via Theorem 4.1, the dual term g* by TopSum, the FISTA loop,
  the Fenchel-dual certificate (§3 "Safe Lower Bound and Pruning"), rounding
  and branching (§4.3).
* ``reopt``   -- re-optimization on a support (§4.3) and brute-force
  enumeration of supports (the definition of problem (intro_sparse_glm)).
* ``bnb``     -- the sequential best-bound branch and bound (Fig. 1 with a
  batch of one node).

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
library routines (LAPACK solves, scipy optimisers and LP), brute force and
invariants (weak/strong duality, Moreau's identity).
"""

from . import losses, node, reopt, bnb  # noqa: F401
