"""Plain, slow, FP64 CPU oracle of the HSDE ADMM for SOS programs
(Zheng, Fantuzzi, Papachristodoulou, "Fast ADMM for sum-of-squares programs
using partial orthogonality").

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke``
and ``bench.py``'s CPU-baseline / reference legs may import it.  The product
path (the CUDA library and its Python binding) never calls into it, and it
shares no code with the product: its conic form, index map, Woodbury solve and
PSD projection are written here independently, following the paper's
equations in its own notation (full ``vec`` Gram columns, eq. (14)).

Modules
-------
basis     monomial bases v_d in graded lexicographic order (eq. (4))
conic     SOS program -> conic data A = [A1 A2 (A3)], b, c, K (eq. (14)-(16),
          eq. (39)-(41))
admm      the three-step ADMM of eq. (20) with the affine step solved by the
          block eliminations of eq. (23)-(28) (Sherman-Morrison + Woodbury),
          cone projection, residuals and termination
dense     dense cross-checks (I+Q) solve for tiny problems
"""

from . import basis, conic, admm, dense  # noqa: F401
