"""Fine-grained DAG execution on one GB300 (sm_103a).

The library proper is ``libdagexec.so`` (C ABI in ``include/dagexec.h``): a
host planner plus one persistent CUDA executor kernel.  This package holds its
sources (``csrc/``), the build step (``build.py``), the ctypes binding
(``_binding.py``, same names as the C ABI), ``dag.py``, a small convenience
layer that turns a workload description into the ABI's structs and moves
numpy arrays in and out, ``spec.py``, the JSON specification frontend
(paper §4.A) with example files in ``specs/``, and ``trace.py``, the export
of a traced launch as a Chrome trace-event file (a Gantt chart per SM).
"""
from . import _binding as abi  # noqa: F401
from .dag import Dag, describe  # noqa: F401
