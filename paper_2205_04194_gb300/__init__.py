"""GB300-native fast inverse-multiquadric matrix-vector product (arXiv 2205.04194).

The compute path is the CUDA library libimq.so (C ABI in include/imq.h);
``paper_2205_04194_gb300.imq`` is its Python binding and
``paper_2205_04194_gb300.workloads`` generates seeded synthetic inputs.
Importing the package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""

__all__ = ["imq", "workloads", "build"]
