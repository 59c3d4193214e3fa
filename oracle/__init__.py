"""FP64 CPU oracle of the ACM-MRT + immersed-boundary kinetic solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may import this package.  The product path
(the CUDA library ``liblbm.so`` and its Python binding) never calls it and shares no
code, table or helper with it; the two only share the seeded input generators in
``scenes``.

It is a plain, slow restatement of the paper's time step (Algorithm 2, Eqs. 1-8) in
float64 with plain PyTorch CPU tensor operations:

* ``lattice``    -- D3Q27 velocities and weights (Eq. 1).
* ``collision``  -- equilibrium, central-moment MRT relaxation with Guo forcing
  (Eqs. 4-5), written twice: literally as Omega = -M^-1 D M (f - f_eq) with an explicit
  27x27 moment matrix solved per node, and with the per-axis (tensor-product) transform.
* ``streaming``  -- two-lattice pull streaming (Eq. 3) with the domain faces.
* ``ib``         -- direct-forcing immersed boundary: interpolation (Eq. 6), penalty
  force (Eq. 7) and spreading (Eq. 8) by scatter and by brute-force gather.
* ``noise``      -- the counter-based SplitMix64 generator of the inlet noise.
* ``solver``     -- the per-step driver in the paper's order (stream, moments, IB,
  collide) and the diagnostics (macroscopic fields, mass/momentum/drag).
* ``adjoint``    -- the loss of the adjoint problem and its exact gradients, obtained
  by reverse-mode differentiation of the FP64 forward step.
* ``motion``     -- prescribed rigid motion of a solid (rotation and translation of its
  samples, boundary velocity), for the moving-solid steps.
* ``tracers``    -- smoke tracers: midpoint-rule advection in the interpolated velocity,
  re-injection, and the cloud-in-cell density projection.

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py`` except
the *adaptive* high-order relaxation rates of ACM-MRT, whose definition lives in
documents the paper defers to and that are not available: parity unpinned for the
adaptive rule; the oracle relaxes orders 3-6 at constant, user-given rates.
"""
