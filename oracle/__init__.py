"""CPU oracle for the SBFEM full-waveform-inversion hot path (TEST INFRASTRUCTURE ONLY).

This package is a plain, slow, FP64 numpy/scipy restatement of what the paper
computes.  It exists to check the CUDA library, never to stand in for it: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference arm
of ``bench.py`` may import it.  It shares no code with the CUDA path
(``paper_2501_06748_gb300``) and imports nothing from it; the only common module
is ``sbfwi_inputs``, which generates seeded inputs and holds none of the method.

Modules, in the order of the paper:

* ``sbfem``      -- Section 3: coordinate map, boundary Jacobian, b1/b2,
  coefficient matrices E0, E1, E2, M0 (Eq. (Es)), radial finite differences and
  the blocks of Eq. (system), the algorithmic condensation (pivots, Thomas sweep,
  last-row elimination, 2x2 closure giving S and the effective source), and the
  back-substitution.
* ``fwi``        -- Section 2 and Section 4: density on nodal points (and the fine
  grid map), Newmark stepping (Eq. (Newmark), Eq. (ODE_Newmark)), the global
  boundary solve, receivers, the misfit (Eq. (misfit)), the time-reversed adjoint
  and the zero-lag cross-correlation kernel with the gradient term dropped.
* ``bruteforce`` -- the full uncondensed element systems of Eq. (system) plus the
  boundary flux balance, solved densely: an independent route to the same
  discrete solution, the pencil for free-vibration frequencies, and the time loop
  on the transposed pencil (source-receiver reciprocity).
* ``modex``      -- the exact derivative of the discrete misfit with respect to the
  nodal densities, by reverse-mode differentiation of the uncondensed time loop
  (pinned by central finite differences); the reference the paper's velocity
  kernel is compared with.
* ``uneven``     -- the condensed path of ``fwi`` on meshes whose elements have
  different numbers of boundary nodes (elements grouped by n_b), with its own
  uncondensed direct solve for pinning.
* ``lfe``        -- Section 3.2: the reduced (constant radial density) equation's
  low-frequency expansion, Riccati stiffness and Lyapunov mass (the paper's
  comparison method), against which the radial finite differences converge.

Parity status of each function is stated in its docstring ("pinned by ..." or
"parity unpinned").
"""
