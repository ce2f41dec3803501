"""GB300 (sm_103a) online all-to-all functional connectivity.

The compute path is the C-ABI library ``libfc.so`` (include/fc.h), hand-written CUDA
for sm_103a; :mod:`paper_2303_03279_gb300.fc` is its thin Python binding.
"""

from . import fc  # noqa: F401
from .fc import Session, FcError, METRIC_BITS  # noqa: F401
