"""FP64 CPU oracle of the Liouville-Lanczos hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import this package.  The product path (the CUDA library and
its Python binding) never imports it and never falls back to it.

It is a plain, slow restatement of the paper's equations in NumPy/SciPy FP64,
sharing no code with the CUDA path:

* ``grid``        -- plane-wave <-> real-space maps (the FFT is a library step).
* ``xc``          -- adiabatic LSDA response kernel f_ab (Eqs. v_XC_q, b_XC_q).
* ``liouvillian`` -- L in the batch representation (Eqs. Liouvillian_BR_q and the
  block actions that follow it, with Eqs. v_H_q, charge_dens_resp_q,
  spin_dens_resp_q, P_minus_q2, P_plus_q2), the end vectors u, v (Sec. 2.5).
* ``lanczos``     -- non-Hermitian biorthogonal and pseudo-Hermitian Lanczos
  recursions (Sec. 2.5).
* ``spectrum``    -- chi(omega) from the tridiagonal matrix (Eqs.
  resolvent_Liouvillian_Lanczos_q and post_processing).

Every function is pinned by a ``-m "not gpu"`` test against something other than
itself (brute-force particle-hole matrices from full diagonalisation, closed
forms, invariants, finite differences, direct DFT sums).  Parity unpinned:
nothing in this package (the mixed-precision error budget lives with the GPU
tests, not here).
"""
