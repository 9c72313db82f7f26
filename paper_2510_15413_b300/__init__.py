"""B300-native engine for the oblivious scan-select of FHE-SQL (arXiv 2510.15413).

The C library (libfhesql.so, interface in include/fhesql.h) holds the TFHE
gate-bootstrap kernels for sm_103a and the scan driver; `fhesql` is its
Python binding and `workloads` the seeded synthetic tables.
"""
from . import fhesql  # noqa: F401
