"""FP64 CPU oracle of the Fullwave 2 time step (arXiv 2106.11476).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or run anything in this
package.  The product path (``paper_2106_11476_gb300``) never touches it, and
the two share no code: the oracle builds its own coefficients from the paper's
closed forms (``oracle.coefficients``), steps the fields with plain C loops
(``fw2_oracle.c`` through ``oracle.core``) and evaluates the paper's analytic
relations (``oracle.analytic``).

Parity status per function (pins live in ``tests/test_oracle_pins.py``):

* relaxation a, b (Eqs. relaxation_a / relaxation_b): pinned by quadrature of
  the kernel zeta and by its DC integral.
* recursion (Eq. relaxation_psi) inside the stepper: pinned by a brute-force
  convolution of the derivative history.
* staggered operator (Sec. 3.1): pinned by exactness on polynomials and by the
  symbol of a sampled sinusoid.
* lossless stepper: pinned by discrete energy conservation and by the
  closed-form discrete dispersion relation.
* attenuating stepper: pinned by the fully discrete dispersion relation of
  the scheme, by the paper's attenuation / phase-velocity claims for its
  Table 2 parameters and by the classical-PML special case.
* C-PML profiles (Sec. 3.3, Table 1): pinned by the normal-incidence
  reflection figures of Sec. 4.2 and by the instability the transition layer
  removes (the counterfactual planted in the oracle grows, the scheme decays).
* nonlinear term (Eq. general6): pinned by the first 7 harmonics of the
  pre-shock Poisson solution of the inviscid Burgers equation (Sec. 4.5),
  with the effective coefficient of each nonlinear mode; the Poisson
  solution itself by the textbook Fubini series.
* Kramers-Kronig target and CFL speed: the y = 1 branch as the limit of the
  general one; c / sqrt(kappa1 kappa2) as the high-frequency limit of the
  dispersion relation.
* staggered-grid placement of rho, kappa, the relaxation parameters and the
  PML coordinate (not printed in the paper): pinned by the discrete energy
  conservation (K with the cell centres, the face density as the mean of the
  two cells), by the echo lag of a face sheet of relaxation parameters
  against the dual centre sheet (a planted upper-cell placement flips it) and
  by the complex-stretching closed form of the C-PML reflection.
* time-space taps (Sec. 3.1): pinned by their dispersion-error orders in 2D
  and 3D and by the Taylor set at r = 0.  The paper's own optimised values are
  not printed: equality with them is parity unpinned.
* relaxation fitter (Sec. 4.1): pinned by the mechanics of the coarse-to-fine
  search and by the paper's 5 % / 0.5 % claims on the polished result of the
  search it restates.  Table 2's
  exact values as the search's result are parity unpinned (the paper states
  neither the reference frequency nor the grid).
* Rusanov reference solver (Sec. 4.5): pinned by the Poisson solution and its
  second-order convergence.
* storage roundings (bf16, FP16 with a power-of-two scale): pinned by bit
  torch's bf16 rounding, numpy's half rounding and idempotence.
"""
