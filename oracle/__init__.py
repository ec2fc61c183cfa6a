"""FP64 CPU oracle for the GRCA hot path (TEST INFRASTRUCTURE ONLY).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It is a plain brute force over all rays
x all triangles written in C (grca_oracle.c); this module only builds and
loads it and marshals numpy arrays.  It never imports the CUDA path.
"""
from .oracle import (MAX_TIES, NO_HIT, Oracle, area_keep, build_oracle, cast, compile_oracle, hit,
                     load_library, range_noise, ray_dirs, ray_tri_margin, splitmix64, triangle_hits)

__all__ = ["MAX_TIES", "NO_HIT", "Oracle", "area_keep", "build_oracle", "cast", "compile_oracle", "hit",
           "load_library", "range_noise", "ray_dirs", "ray_tri_margin", "splitmix64", "triangle_hits"]
