"""FP64 CPU oracle for finite-temperature CCSD (White & Chan, arXiv:2004.01729).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library in
``paper_2004_01729_gb300/`` (no kernels, helpers, tables or constants); the
only common module is the seeded input generator
``paper_2004_01729_gb300/workloads.py``, which holds no FT-CC arithmetic.

Contents
  systems.py  model Hamiltonians (1D Hubbard in k space, in the site basis
              with the Neel-state or UHF reference, plane-wave UEG, generic), built
              from their textbook definitions; the staggered magnetisation
              of a site-basis 1-RDM.
  ftccsd.py   reference quantities, thermal integrals (App. A), the Simpson
              quadrature tensors (Sec. II.C, Eqs. g/G), the E, S1, S2
              kernels term by term (Eqs. E, ccS1, ccS2), the integral-form
              fixed point (Eq. smu / Alg. 2), the lambda equations (Eqs.
              Lagrangian, lmu, ltilde) and response outputs (App. B).
  differential.py  the differential form of the amplitude equations (Eq.
              smud) marched over the grid by explicit RK1 / RK2 / RK4 steps
              (Alg. 1), with Omega_CC from the same quadrature weights.
  chemical_potential.py  the chemical potential for a fixed mean particle
              number: the reference mu_0 (Fermi sum) and mu_CC from the
              FT-CCSD N(mu) = -dOmega/dmu (App. B, App. D).
  exact.py    exact grand potentials (Fock-space diagonalisation and
              non-interacting closed forms) used only to pin the oracle.

Every function is plain and slow by design; torch is used on the CPU in
float64 so that reverse-mode differentiation is available for the lambda
equations and the property derivatives.
"""
