"""FP64 CPU oracle for the DG thermal-noise path (arXiv 2111.06893).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library and the library never calls it.

It is a plain, slow restatement of the paper's method:

* ``lgl``          LGL nodes, weights and the Lagrange basis (Sec. 2.2.1)
* ``mesh``         box and cylinder decomposition, element maps, Jacobians
                   by complex step, neighbours found from coordinates
* ``materials``    Eqs. (constrel_iso), (constrel_cryst)
* ``dg``           explicit element matrices of the DG operator
                   (Sec. 2.2.2-2.2.4), assembled; the paper's strong form too
* ``observables``  direct solve, per-layer energies, Eq. (thermalnoise),
                   the half-space closed form
* ``gradient``     derivatives of the energies by complex step through the
                   whole oracle computation

Every function cites the passage it follows.  Parity status of each part is
listed in the design notes; the readings where the paper is silent are the
ones stated in the module docstrings.
"""
from .dg import Operator
from .mesh import Mesh
from . import observables

__all__ = ["Mesh", "Operator", "observables"]
