"""FP64 CPU oracle for the implicit momentum-conserving APIC-MPM step with
spatially varying surface energy (arXiv 2101.12408).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The CUDA library never calls it and shares no code with it.

Plain, slow, obviously checkable numpy in float64. Each function names the
section / equation of the paper it follows. Readings taken where the paper is
silent or garbled are written next to the code that uses them.
"""
from .spline import Stencil, axis_weights, node_positions, scatter, gather  # noqa: F401
from .resample import nearest_parent, split  # noqa: F401
from .transfer import p2g, g2p, grid_velocity  # noqa: F401
from .boundary import projector, apply_projector  # noqa: F401
from .constitutive import cof, dcof, levi_civita, polar, fcr_energy, fcr_P, fcr_dP  # noqa: F401
from .energy import NewtonState  # noqa: F401
from .heat import HeatSystem  # noqa: F401
from .solver import newton_solve, pcg, heat_solve  # noqa: F401
from .step import OracleSim  # noqa: F401
