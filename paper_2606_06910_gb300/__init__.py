"""GB300-native radius-4 acoustic FDTD with CPML (paper Sec. 3.1-3.2).

``Fdtd`` / ``FdtdFn`` (module ``fdtd``) wrap the CUDA library declared in
include/fdtd.h; ``LearnedCPML`` (module ``learned``) trains the learned CPML
grading with the library's kernels; ``synth`` holds the seeded input
generators.  Importing the package loads neither torch nor the library; the
library is built and loaded on first use.
"""

__all__ = ["Fdtd", "FdtdFn", "FdtdError", "LearnedCPML"]


def __getattr__(name):
    if name in ("Fdtd", "FdtdFn", "FdtdError"):
        from . import fdtd
        return getattr(fdtd, name)
    if name == "LearnedCPML":
        from . import learned
        return learned.LearnedCPML
    raise AttributeError(name)
