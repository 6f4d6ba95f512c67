"""B300-native (sm_103a) FKS two-level static hash maps.

Build and query Fredman-Komlos-Szemeredi two-level, collision-free hash maps
(Due, Elsman, Henriksen, arXiv 2508.11443) with hand-written CUDA kernels
behind the C ABI declared in ``include/fks.h``.

* ``paper_2508_11443_b300.fks``        ctypes binding of the C ABI (same names)
* ``paper_2508_11443_b300.build``      in-tree nvcc build of ``libfks.so``
* ``paper_2508_11443_b300.workloads``  seeded synthetic inputs of the benchmarks

The binding is imported lazily so that the input generators can be used on a
machine without the compiled library.
"""
