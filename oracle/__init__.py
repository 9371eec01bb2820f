"""Plain, slow FP64 CPU oracle for the symmetry-reduced BSE block builder.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA library and never imports it; the library
never imports this package.

It follows the definitions of Stöhler, Blügel and Friedrich, "Efficient
all-electron Bethe-Salpeter implementation using crystal symmetries":
  * tables        - symmetry operations, k stars, characters (Sec. III.C)
  * hamiltonian   - pair densities, exchange, direct term, head correction,
                    full H (Eqs. BSE-eigval, w_interaction, w_interaction2,
                    Wdiv, divergence_int, divergence_sum)
  * projection    - band rotations, two-particle representation, projector,
                    orbit-wise orthonormal basis, H_mu (Eqs. Ts, Ttilde,
                    projection, transformationU)
  * spectrum      - block eigensolution, oscillator strengths, Im eps_M
                    (Eqs. macro_diel, reducible_polar, oscillatorA, oscillator)
  * loss          - longitudinal excitons and the loss spectrum (Eqs. secular,
                    eigenvec_xi, epsinv_div)
  * haydock       - Lanczos-Haydock spectrum of a block (Sec. IV): Lanczos
                    recurrence and continued fraction

Functions whose result has no independent pin say "parity unpinned" in their
docstring.  At present every function has at least one pin in tests/.
"""
