"""Plain FP64 CPU oracles of the DG Euler hot path (test infrastructure).

This package is the independent check of the CUDA library: slow, written for
reading, in float64 numpy. It is used only by the tests, by the bench's CPU
baseline leg and by the smoke check; the library never imports it, and it
imports nothing from the library (its only shared input is the seeded
workload module, which holds no DG arithmetic).

Modules:
  reference_element  nodes, interpolation, derivative / mass / lift matrices
                     (Appendix A, Eqs. 10-11), built from a monomial basis with
                     exact integrals
  geometry           affine maps, normals, face matching by coordinates
  euler_dg           Euler fluxes (Eqs. 1-2), boundary ghost states (free
                     stream, characteristic, wall: sections 2.2-2.3, Eq. 4;
                     inflow pulse: section 2.4, Eqs. 5-7; the learned closure
                     and its spherical-wave memory), local Lax-Friedrichs
                     flux, semi-discrete right-hand side (Eqs. 10, 12) and its
                     contraction inputs, low-storage RK4, probes,
                     boundary-flux ledger and conserved totals
  mlp                the closure's network (forward, loss gradient, Adam) and
                     its features
  modal_dg           the paper's own discretisation (Appendix A): orthonormal
                     basis, Gauss quadrature of degree 2p / 2p+1 for Eq. 10,
                     Heun's RK2
"""
