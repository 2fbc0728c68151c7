"""FP64 CPU oracle of the diffuse-interface LB freezing step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never does, and this
package imports nothing from it.

The C source ``lb_oracle.c`` is compiled with gcc into ``liblboracle.so`` next
to it (``build_oracle()``), without fast-math and with FMA contraction off.
"""
from .oracle import (GRID_FIELDS, PARAM_FIELDS, Oracle, build_oracle, enthalpy_forward,
                     enthalpy_invert, equilibria, lib, sources, stencil_field, zeta)

__all__ = ["GRID_FIELDS", "PARAM_FIELDS", "Oracle", "build_oracle", "enthalpy_forward",
           "enthalpy_invert", "equilibria", "lib", "sources", "stencil_field", "zeta"]
