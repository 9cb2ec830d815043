"""GB300-native fast spectral Boltzmann collision operator (arxiv 2505.03360 hot path).

Modules:
  coll     ctypes binding of libcoll.so (the C ABI of include/coll.h); importing it
           requires the built library and raises otherwise (no CPU fallback)
  synth    seeded synthetic inputs (shared by tests, bench and the oracle)
  build    in-tree nvcc build of libcoll.so for sm_103a
  service  continuous-batching request loop over the C ABI
"""
