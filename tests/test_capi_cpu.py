"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and the ctypes mirrors of the public structs have the C layout.
No compute call is made (there is no GPU here)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rism3d.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"RISM_API\s+[\w\s\*]*?\b(rism_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2109_09772_gb300 import build as B

    B.build()
    from paper_2109_09772_gb300 import rism

    return rism.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("rism_grid_create", "rism_set_solute", "rism_set_solvent", "rism_potential", "rism_asymptotics",
              "rism_potential_backward"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2109_09772_gb300 import rism

    names = _declared()
    assert sorted(rism.EXPORTS) == sorted(n for n in names if n in rism.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", rism.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rism_\w+)", out))
    assert set(names) <= exported
    # nothing else leaks out of the library
    assert exported <= set(names)


def test_struct_layout_matches_c(lib):
    from paper_2109_09772_gb300 import rism

    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "rism3d.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(rism_grid_desc), sizeof(rism_options), sizeof(rism_info),
         offsetof(rism_options, wait_limit), offsetof(rism_options, debug_flags), offsetof(rism_info, batch),
         offsetof(rism_options, theta));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    assert vals == [C.sizeof(rism.GridDesc), C.sizeof(rism.Options), C.sizeof(rism.Info),
                    rism.Options.wait_limit.offset, rism.Options.debug_flags.offset, rism.Info.batch.offset,
                    rism.Options.theta.offset]


def test_default_options_without_gpu(lib):
    from paper_2109_09772_gb300 import rism

    o = rism.default_options()
    assert o.method == rism.METHOD_TREECODE and o.precision == rism.PREC_FP32
    assert o.degree == 8 and abs(o.theta - 0.7) < 1e-15 and o.lj_mode == rism.LJ_RCUT and o.lj_rcut == 9.0
    assert o.eta == 1.0 and o.T == 298.0 and o.kappa == -1.0 and o.wait_limit > 0


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_2109_09772_gb300 import rism

    o = rism.default_options()
    ctx = C.c_void_p()
    # NULL descriptor / output pointer, and bad grids, are rejected before any CUDA call
    assert lib.rism_grid_create(None, C.byref(o), None, C.byref(ctx)) == rism.E_INVALID
    g = rism.GridDesc(0, 4, 4, 0.5, (C.c_double * 3)(0, 0, 0))
    assert lib.rism_grid_create(C.byref(g), C.byref(o), None, C.byref(ctx)) == rism.E_INVALID
    g = rism.GridDesc(4, 4, 4, -0.5, (C.c_double * 3)(0, 0, 0))
    assert lib.rism_grid_create(C.byref(g), C.byref(o), None, C.byref(ctx)) == rism.E_INVALID
    g = rism.GridDesc(4, 4, 4, 0.5, (C.c_double * 3)(float("nan"), 0, 0))
    assert lib.rism_grid_create(C.byref(g), C.byref(o), None, C.byref(ctx)) == rism.E_INVALID
    g = rism.GridDesc(4, 4, 4, 0.5, (C.c_double * 3)(0, 0, 0))
    bad = rism.default_options(theta=1.5)
    assert lib.rism_grid_create(C.byref(g), C.byref(bad), None, C.byref(ctx)) == rism.E_INVALID
    bad = rism.default_options(degree=0)
    assert lib.rism_grid_create(C.byref(g), C.byref(bad), None, C.byref(ctx)) == rism.E_INVALID
    # the treecode computes FP32 pair terms: asking it for FP64 is refused, not silently downgraded
    bad = rism.default_options(method=rism.METHOD_TREECODE, precision=rism.PREC_FP64)
    assert lib.rism_grid_create(C.byref(g), C.byref(bad), None, C.byref(ctx)) == rism.E_UNSUPPORTED
    # NULL contexts
    assert lib.rism_init(None, None, None, None, None) == rism.E_INVALID
    assert lib.rism_set_solute(None, 0, None, None, None, None) == rism.E_INVALID
    assert lib.rism_last_error(None) is not None
    lib.rism_destroy(None)
