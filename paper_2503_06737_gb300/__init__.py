"""GB300-native (sm_103a) CS/HCS LSH hashing and indexing.

Implements the hot path of "Faster and Space Efficient Indexing for Locality
Sensitive Hashing" (arXiv 2503.06737): CS-E2LSH, HCS-E2LSH, CS-SRP and HCS-SRP
hashcodes for all L tables in one launch, the dense E2LSH/SRP baseline, the
hash-table index and the query path, behind the C ABI of include/lsh.h.

`lsh` is the ctypes binding of that ABI; `workloads` draws seeded synthetic
inputs; `build` compiles the CUDA library in-tree.
"""
from . import lsh  # noqa: F401
from .lsh import Family, Index, LshError  # noqa: F401
