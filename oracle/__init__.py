"""FP64 CPU oracle for the semi-Lagrangian lattice Boltzmann (SLLBM) step of arXiv:1910.13918.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` use it.  It shares no code with the CUDA library or its Python binding and imports
nothing from them.

Modules
-------
``sllbm``    velocity set, Hermite equilibrium, grid, departure points, streaming, collision,
             diagnostics (Sec. II of the paper), written as plain loops in float64.
``sllbm3d``  the same step in three dimensions (D3Q125 on hexahedral cells), reusing the
             dimension-free parts of ``sllbm``.
``adjoint``  reference adjoint of one step: complex-step collision Jacobian and a scatter
             transpose of the interpolation.
``riemann``  exact Riemann solver for the Euler equations (validation of the Sod case, Sec. III.C).

Parity status of every function is recorded in its docstring; all are pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
