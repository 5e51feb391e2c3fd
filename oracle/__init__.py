"""Plain FP64 CPU oracle for the volumetric lattice Boltzmann method for
thermal particulate flows with conjugate heat transfer (Zhang, Wang, Li,
Huang, arXiv 2410.23802).

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline / reference legs of
``bench.py`` and by nothing else.  The product path (the CUDA library and
its Python binding) never imports, links or executes anything here, and this
package imports nothing from the product.

Every function cites the equation or section of the paper it writes out.
Readings of passages where the paper is silent are listed in the module
docstring of :mod:`oracle.vlbref`.

Parity status: every function is pinned by a ``-m "not gpu"`` test (the
momentum-exchange force and torque by the linear and angular momentum
balances of every step and by Stokes drag and torque; the buoyancy and the
joint temperature/velocity solve by exact buoyant Poiseuille, conduction-slot
and stratified-layer states), except the fully coupled many-step trajectory
(flow + heat + particles), for which no closed form exists: "parity
unpinned" beyond the invariants (mass, energy bookkeeping, isothermal
invariant of Appendix A, u = u_s in solid cells, Galilean zero force, the
momentum balances) that the tests check on coupled runs.
"""
from .vlbref import *  # noqa: F401,F403
