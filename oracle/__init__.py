"""CPU FP64 oracle of the low-rank all-at-once solver (Elman & Su).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py may import this package; the GPU library never does,
and shares no code, tables or helpers with it.  Inputs come from `synth`
(geometry, viscosity model, conventions), which holds no solver arithmetic.

Modules and the passages they follow:
  fem     Q2-Q1 matrices, eq. (mat_entries) and the divergence B (Section 3.2)
  gpc     G_l, H_l (Section 3.2), Legendre chaos (Section 5.1)
  tt      tensor trains, eq. (z_tt), eq. (Xz), Algorithm 4.1, truncation (Section 4.1)
  system  the all-at-once operator, eq. (F), eq. (ns_sys_all), eq. (N_kron)
  solver  Algorithm 4.2, eq. (mean_lsc), eq. (11_prec), Algorithm 3.1
  learned the learned replacement of K^{-1} in eq. (11_prec) (no counterpart in
          the paper): conv net forward/backward, loss, Adam, training pairs

Every function is pinned by a `-m "not gpu"` test to something other than
itself (closed forms, exactly representable solutions, a sparse direct solve
of the uncompressed system, the paper's printed sizes); see tests/test_oracle_*.
"""
