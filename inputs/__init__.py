"""Seeded synthetic inputs shared by the CUDA path's tests and bench and by the
oracle.

This package holds none of the method's arithmetic (no equation of state
evaluation of the solver, no derivatives, no assembly, no time stepping): it
only samples analytic fields at node positions and draws seeded random numbers.
Both sides receive the same arrays from here; nothing here imports the oracle
or the library.

* ``rng``        -- SplitMix64, a counter-based 64-bit generator (Steele, Lea &
                    Flood 2014), written from its published definition.
* ``grid``       -- node positions of the box meshes (LGL points via numpy's
                    Legendre-series roots; a third, independent construction).
* ``atmosphere`` -- reference soundings, the rising-bubble and warm-core-vortex
                    initial states, the synthetic heating field and seeded
                    smooth random states.
* ``workloads``  -- the named workloads (sizes, parameters, recipes).
"""

from . import rng, grid, atmosphere, workloads  # noqa: F401
