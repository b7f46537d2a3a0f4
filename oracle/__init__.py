"""CPU FP64 oracle for the MDP projection columns -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct restatement of what the hot path computes
(North, Tsynkov & Turkel, Sections 3.1-3.2): it assembles the sparse
auxiliary-problem (AP) matrix, factors it with SuperLU (scipy.sparse.linalg.splu),
and forms each projection column with one sparse solve.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
leg and ``--impl reference``) may import this package. The CUDA library never
imports, links or executes anything here, and this package shares no code,
table or constant generator with it; the only shared module is ``workloads``
(seeded input descriptions, no arithmetic of the method).

Modules:
  grid        -- grid sets N0, M0, M+, M-, N+, N-, gamma; side ownership (Section 3.2.2)
  scheme      -- compact 9-point operator and AP matrix (Section 3.1, 3.2.1)
  extension   -- Chebyshev basis and equation-based extension (Sections 3.2.3-3.2.4)
  projection  -- G^(h), P_gamma, Q columns, adjoint, wavenumber gradient (Sections 3.2.2, 3.2.5)
  dd          -- multi-subdomain coupling for the layered strip (Sections 3.3-3.5)

Parity status: every function is pinned by tests under tests/test_oracle_*.py
except the ones whose header says "parity unpinned".
"""
