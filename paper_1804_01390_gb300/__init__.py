"""GB300-native (sm_103a) reflectionless discrete PML (Chern, arXiv 1804.01390).

The compute path is the C-ABI library ``libpml.so`` (``include/pml.h``), built from
``csrc/`` by ``build.py``.  ``_lib`` binds its entry points one to one;
``solver.PMLSolver`` adds torch device memory and streams; ``autograd`` exposes the
hand-written adjoint as a ``torch.autograd.Function``; ``workloads`` draws the seeded
synthetic inputs.  Importing the package does not load the library (so the seeded
input generators work without a GPU); the first call that needs it loads it and
fails loudly if it has not been built.
"""

__all__ = ["PMLSolver", "PMLBatch"]


def __getattr__(name):
    if name == "PMLSolver":
        from .solver import PMLSolver
        return PMLSolver
    if name == "PMLBatch":
        from .solver import PMLBatch
        return PMLBatch
    raise AttributeError(name)
