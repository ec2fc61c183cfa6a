"""GB300-native GRCA (emitter-centric LiDAR ray casting) — Python side.

`grca` is the ctypes binding of libgrca.so (C ABI in include/grca.h); `build`
compiles the library for sm_103a.  Importing this package does not load the
library; constructing a `grca.Caster` does, and fails loudly without it.
"""
__all__ = ["grca", "build"]
