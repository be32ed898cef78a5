"""GB300-native renderer of a dynamic human from a canonical radiance field.

Submodules:
  synth  seeded synthetic inputs (skeleton, poses, cameras, volumes, tables)
  build  compiles csrc/*.cu into libnr.so for sm_103a
  nr     ctypes binding of libnr.so (the C ABI of include/nr.h)

`nr` is imported on demand so that the input generator is usable without
the compiled library.
"""
__all__ = ["synth", "build", "nr"]
