"""CPU oracle for the evaporation operators — TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct float64 implementation of what the GPU hot path computes, written from the paper
(Schreter-Fleischhacker et al., "A consistent diffuse-interface model for two-phase flow problems with rapid
evaporation", arXiv 2401.07805).  Element matrices are formed by full Gauss quadrature of the weak forms (App. D)
and assembled into sparse matrices; nothing is sum-factorised, fused or reordered.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``
may import this package.  The product library never calls it and shares no code with it.

Modules:
  fe         1D Lagrange bases on Gauss-Lobatto points, Gauss-Legendre rules, 3D tensor bases, mesh connectivity
  physics    per-point material law: Heaviside, delta, reciprocal density, viscosity, normal, dilation rate
  momentum   linearized momentum operator (velocity block) and the divergence row with evaporation source
  levelset   level-set advection (Crank-Nicolson) and conservative reinitialization operators
  transport  transport velocity variants 1/2/3 with closest-point projection (App. C)
  adjoint    transposed operator and parameter gradients of w.A(phi, mdot, u0)x + w_p.(Bx - g)
  solve      direct sparse solve of the momentum system (definition of the solution)
"""
from . import fe, physics, momentum, levelset, transport, adjoint, solve  # noqa: F401
