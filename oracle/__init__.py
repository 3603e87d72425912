"""Plain FP64 CPU oracle for the kagome DQMC time-slice sweep.

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (the CUDA library under ``paper_2608_03894_gb300/`` and its
Python binding) never imports, links or calls anything here, and the two share
no code: no kernels, tables, constants or pre/post-processing. The only module
both sides use is ``dqmc_inputs`` (seeded synthetic inputs, no method
arithmetic).

What the oracle computes, and where each piece comes from
(arXiv 2608.03894, "Accelerated quantum Monte Carlo simulations of the
attractive Hubbard model on the kagome lattice"):

* ``lattice``  -- the kagome kinetic matrix K built literally from its
  Kronecker form (Sec. II, Eq. 3), the Fourier block-diagonalisation of
  Eq. 2 / Eq. 4 and the three-step FFT propagator product of Eq. 5-6.
* ``philox``   -- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the
  counter-based generator both sides implement from its published definition.
* ``model``    -- the Hamiltonian of Eq. 1 (U < 0 is attraction), its
  discrete charge-channel Hubbard-Stratonovich decoupling and the slice
  propagators B_l = e^{V_l} e^{-dtau K} (dense, exp by eigendecomposition).
* ``green``    -- the equal-time Green's function from scratch: direct
  inversion, and the UDV (column-pivoted QR) scale-separated inversion.
* ``dqmc``     -- the Metropolis sweep with one-at-a-time Sherman-Morrison
  updates, dense wraps and periodic UDV recomputation.
* ``measure``  -- Wick-contracted s-wave pair structure factor (Sec. III,
  symmetric definition), the CDW field correlator of Sec. IV, density and
  kinetic energy.
* ``fock``     -- exact diagonalisation and Fock-space Trotter products on
  tiny tori (3 and 6 sites), and the brute-force sum over all HS fields.
* ``lattices`` -- the other composite lattices of the appendix: the
  triangular (1 x 1 blocks) and honeycomb (2 x 2 blocks) kinetic matrices
  from their Kronecker forms and from geometry.
* ``pqmc``     -- the projector (zero-temperature) variant of the paper
  (Sec. II): trial Slater determinant from the lowest N_occ eigenstates of
  K, G = I - R (L R)^{-1} L from orthonormal N x N_occ stacks, the same
  sweep and proposals.

Pins (tests marked ``not gpu``) tie every function to something other than
itself: the textbook kagome band structure, scipy's Pade ``expm``, the U=0
closed form, the exact HS/Trotter identity in Fock space, Delta-tau^2
convergence to exact diagonalisation, an exact-weight histogram of the Markov
chain, and the Philox known-answer vectors.
"""

from . import lattice, lattices, philox, model, green, measure, fock, dqmc, pqmc  # noqa: F401
