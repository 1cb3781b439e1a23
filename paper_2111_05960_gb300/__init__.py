"""GB300-native coupled phi-mu lattice Boltzmann step of the grand-potential
phase-field model of dissolution/precipitation (arXiv 2111.05960).

The compute path is libgb_lbpf.so (hand-written CUDA for sm_103a behind the C
ABI of include/lbpf.h); ``lbpf`` is its thin ctypes binding and ``workloads``
builds seeded synthetic inputs.
"""
from . import workloads  # noqa: F401


def binding():
    """The ctypes binding module, with libgb_lbpf.so loaded."""
    import importlib
    b = importlib.import_module(__name__ + ".lbpf")
    b.load()
    return b
