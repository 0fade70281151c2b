"""CPU oracle for the MGRIT eddy-current machine path — TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 NumPy/SciPy code that states what the GPU library computes,
written from the paper (Bolten, Friedhoff, Hahne, Schoeps, "Parallel-in-Time
Simulation of an Electrical Machine using MGRIT", arXiv:1912.03106):

  fem.py       P1 assembly of the semi-discrete system M a' + K(a) a = f  (Sec. 3.1,
               Eq. semi_discrete_system), Dirichlet elimination, Brauer-law Jacobian
  pwm.py       three-phase PWM switching functions (Sec. 3.2-3.3, Eqs. machine_pwm,
               machine_reference_signal, machine_carrier_signal)
  stepper.py   backward-Euler propagator Phi and the sequential forward block solve
               (Sec. 2, Eq. mgrit_nonlinear_system and the block-bidiagonal system;
               Sec. 3.1 Eq. discrete_system), Newton for the nonlinear law (Sec. 5)
  transfer.py  P1 nodal-interpolation prolongation between nested meshes and the
               spatial restrictions (Sec. 3.4, Sec. 2.2)
  mgrit.py     FAS-MGRIT, Algorithm 1 with F/FCF relaxation, injection, ideal
               interpolation, spatial coarsening and the recursive V-cycle (Sec. 2.1-2.2)
  scalar.py    scalar test propagators for the two-level error closed form

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg
may import this package.  It shares no code with the CUDA library; its only
inputs are the seeded data of the `synth` package.
"""
