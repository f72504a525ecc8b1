"""CPU oracle for the QML / pixel-likelihood hot path (TEST INFRASTRUCTURE ONLY).

This package is a plain, slow, double-precision restatement of what the method
computes, written from the paper's definitions.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import it; the CUDA library and
its Python binding never do, and it never imports them.  It shares no code with
the CUDA path: the only common module is the seeded input generator, which
holds none of the method's arithmetic.

Modules
  wigner   small Wigner d-matrix: d = exp(-i beta J_y) (definition) and the
           textbook factorial sum (for pins on small l)
  harmonic real spin-0 / spin-2 harmonic matrix Y (pixels x modes) with the
           transfer function folded in (Eqs. addition_theorem, real_ylm;
           App. A, Eqs. spin_y_def, EB_from_spin)
  qml      Fisher matrix, noise bias, quadratic estimates, the three
           normalisations and the pixel likelihood by their definitions
           (Sect. 2.2, 2.3.3, 2.5, 2.6)
  brute    dense pixel-space derivatives P_a built from Legendre sums and
           complex spin-weighted harmonic pair sums, for tiny inputs

Every function is pinned by a `-m "not gpu"` test to something other than
itself (closed forms, textbook values, brute force, invariants); there is no
"parity unpinned" function.
"""
