"""CPU tests: the FP64 oracle against its pins, and planted mistakes.

The planted-mistake test copies the oracle source, plants one plausible
mistake (a flipped sign, a dropped term, a wrong comparison), compiles the copy
into a temporary library and checks that at least one pin fails on it.
"""
import os
import shutil
import tempfile

import pytest

import oracle
from oracle.oracle import HERE as ORACLE_DIR
from oracle.oracle import SRC as ORACLE_SRC

import oracle_pins as pins


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda f: f.__name__)
def test_pin(check):
    check()


MUTANTS = [
    ("right axis sign in Eq. ray_dir", "+ b * s->r[k]", "- b * s->r[k]"),
    ("elevation term dropped from Eq. ray_dir", "+ c * s->u[k]", "+ 0.0 * s->u[k]"),
    ("cos/sin swapped in azimuth", "double a = cos(th) * cos(ph), b = sin(th) * cos(ph)",
     "double a = sin(th) * cos(ph), b = cos(th) * cos(ph)"),
    ("inside test inverted", "if (dot3(c, n) < 0.0) return 0;", "if (dot3(c, n) > 0.0) return 0;"),
    ("edge index off by one", "const double* b = V[(k + 1) % 3];\n        double ab[3], ax[3], c[3];",
     "const double* b = V[(k + 2) % 3];\n        double ab[3], ax[3], c[3];"),
    ("t numerator sign flipped", "sub3(v0, o, w);\n    double t", "sub3(o, v0, w);\n    double t"),
    ("t denominator dropped", "double t = dot3(n, w) / denom;", "double t = dot3(n, w);"),
    ("ties keep the higher id", "&& t < best)", "&& t <= best)"),
    ("facing rule sign", "return dot3(n, w) > 0.0;", "return dot3(n, w) < 0.0;"),
    ("d_max not applied", "if (tt < s->d_min || tt > s->d_max) return 0;", "if (tt < s->d_min) return 0;"),
    ("channel index taken from the ray index", "double ph = s->elev[j];", "double ph = s->elev[i % s->n_channels];"),
    ("behind-origin hits accepted", "if (!(t > 0.0)) return 0;", "if (t == 0.0) return 0;"),
    ("transposed cross product operands", "cross3(ab, ax, c);", "cross3(ax, ab, c);"),
    ("apparent-area threshold not squared", "double rhs = eps * eps * r2 * r2 * r2;", "double rhs = eps * r2 * r2 * r2;"),
    ("Box-Muller radius without the factor 2", "z[k] = sqrt(-2.0 * log(u1))", "z[k] = sqrt(-log(u1))"),
    ("SplitMix64 second shift wrong", "z = (z ^ (z >> 27))", "z = (z ^ (z >> 28))"),
    ("both uniforms from the same counter", "double u2 = (double)(orc_splitmix64(c + 1ull) >> 40)",
     "double u2 = (double)(orc_splitmix64(c) >> 40)"),
    ("listed azimuth taken from the channel index", "double th = s->theta ? s->theta[i]",
     "double th = s->theta ? s->theta[j % s->n_rays]"),
    ("ray mask bit order reversed", "if (s->mask && !((s->mask[q >> 5] >> (q & 31u)) & 1u)) {",
     "if (s->mask && !((s->mask[q >> 5] >> (31u - (q & 31u))) & 1u)) {"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new):
    src = open(ORACLE_SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    tmp = tempfile.mkdtemp(prefix="orc_mut_")
    try:
        p = os.path.join(tmp, "grca_oracle.c")
        open(p, "w").write(src.replace(old, new))
        shutil.copy(os.path.join(ORACLE_DIR, "grca_oracle.h"), tmp)
        lib = oracle.load_library(oracle.compile_oracle(p, os.path.join(tmp, "libmut.so"), tmp))
        failed = []
        for check in pins.ALL_CHECKS:
            try:
                check(lib)
            except (AssertionError, ValueError):
                failed.append(check.__name__)
        assert failed, f"planted mistake '{name}' passed every pin"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
