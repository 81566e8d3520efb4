"""Plain FP64 CPU oracle for the density-fitted PNOF7 JK step (test infrastructure only).

This package is the slow, obviously correct restatement of what the GPU library computes.
It exists to check the CUDA path; only the test suite, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import it. The product path never
calls it and never falls back to it.

It shares no code with the CUDA path: both consume the seeded inputs of
`paper_2512_13550_gb300.inputs` (random numbers, geometries, basis specifications), and
nothing else.

Modules and the passages they follow (DoNOF 2.0, arXiv 2512.13550):
  integrals  one- and two-electron integrals over s Gaussians (Theory section, the definitions
             of h_ki and <kl|ij>); the closed forms are the textbook s-Gaussian formulas.
  ri         resolution-of-the-identity (density-fitted) three-index tensor B^P_{mu nu}
             (Single Point Energy section, ERITYP='RI').
  pnof       pairing structure (Eq. OmegaG, Eq. sum1, Fig. 1), trigonometric ON mapping
             (Occupation Number Optimization subsection), the JKL-only energy (Eq. PNOF),
             the Lagrangian and the orbital gradient g = 4(lambda - lambda^T)
             (Natural Orbital Optimization subsection).
  step       ADAM orbital-rotation step C <- C exp(y) and the ON update.
  reference  brute-force validators for tiny systems: exact 4-index ERIs, RHF in AO form,
             two-electron full CI, two-orbital DOCI.
  rdm        the reconstructed spin-orbital 2RDM of the cumulant expansion (Theory section,
             the Delta/Pi structure) and Eq. (Energy) contracted with it: a second route to
             the energy that pins the A/B bookkeeping of pnof.

Parity status per function is recorded in each module header. Functions whose result the
paper does not fix (the PNOF7 A/B coefficients and the ADAM hyper-parameters, which the paper
delegates to other publications) are marked there as readings.
"""
