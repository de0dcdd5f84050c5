"""FP64 CPU oracle for symmetry-masked autoregressive VMC (arXiv:2310.04166).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of what the paper's method computes.  It exists to
check the CUDA library; it is imported only by ``tests/``, by the smoke check
in ``__graft_entry__`` and by the CPU-baseline leg of ``bench.py``.  The
product path (``paper_2310_04166_gb300``) never imports it and shares no code
with it; the only shared module is ``synthetic`` (seeded random inputs, no
method arithmetic).

Modules, each citing the passage it follows:

* ``philox``      Philox4x64-10 counter-based generator (Salmon et al., SC'11).
* ``sector``      Quantum-number symmetries and IsPhys (Sec. III.B, Alg. 1,
                  Proposition 1, Appendix A).
* ``hamiltonian`` Second-quantised Hamiltonian (Eq. sq_hamiltonian), Jordan-
                  Wigner signs (Sec. IV.A), Slater-Condon elements, the dense
                  JW Pauli-product matrix and the connected set of a sample.
* ``anqs``        Autoregressive ansatz (Eq. anqs_def), per-slot MLP (Appendix
                  B.1) and causal transformer, MU masking (Sec. III.C), tabular
                  ansatz built from a given state.
* ``sampler``     Autoregressive statistics sampling with MU (Sec. II.C,
                  Sec. III.C).
* ``vmc``         Local energy (Eq. local_energy_def), count-weighted energy
                  (Eq. energy_est), variance, gradient (Eq. grad_def).
* ``ed``          Exact diagonalisation of a sector (for pins only).

Pinned in ``tests/test_oracle_*.py``; every function without such a pin says
"parity unpinned" in its docstring.
"""
