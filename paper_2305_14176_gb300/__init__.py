"""GB300 (sm_103a) FMCW radar simulation from ray-tracer output and meta data.

The compute path is the C ABI of ``libradarsim.so`` (see include/radarsim.h);
``radarsim`` is its ctypes binding.  Importing this package loads the library
and raises if it has not been built.
"""
from . import radarsim  # noqa: F401
from .radarsim import Context, SimError  # noqa: F401
