"""FP64 CPU oracle for the connectivity hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg
of ``bench.py`` may import this package. The product path (the CUDA library and
its Python binding) never imports, calls or links anything in here, and this
package imports nothing from the product path.
"""

from .fc_oracle import *  # noqa: F401,F403
