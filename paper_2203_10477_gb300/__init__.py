"""RSWR (arXiv 2203.10477) on GB300: the data-parallel hot path as CUDA kernels
behind a small C ABI (include/rswr.h), with a thin Python binding.

Submodules: ``rswr`` (binding), ``build`` (nvcc build), ``inputs`` (seeded
synthetic workloads).  Importing the package does not load the library.
"""
