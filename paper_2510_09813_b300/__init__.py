"""B300-native state-vector emulator for Rydberg atom arrays (arXiv 2510.09813).

The compute path is the CUDA library librsv.so (C ABI in include/rsv.h);
`paper_2510_09813_b300.api` is its thin Python front end and
`paper_2510_09813_b300.workloads` generates seeded synthetic inputs.

Importing the package does not load the CUDA library; `api` functions load it
on first use and raise if it has not been built.
"""

__all__ = ["api", "workloads"]
