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


def _noalloc_args(rism, n=3, **over):
    """Arguments of a valid rism_init_noalloc call on host arrays, with one field replaced."""
    import numpy as np

    a = dict(grid=rism.GridDesc(8, 8, 8, 0.5, (C.c_double * 3)(-1.75, -1.75, -1.75)),
             opts=rism.default_options(method=rism.METHOD_DIRECT), n=n,
             xyz=np.zeros((n, 3)), q=np.ones(n), sigma=np.full(n, 2.0), eps=np.full(n, 0.1),
             qs=np.array([-0.8, 0.4]), sigs=np.array([3.0, 1.0]), epss=np.array([0.15, 0.01]),
             rho=np.array([0.03, 0.06]))
    a.update(over)
    return a


def _call_noalloc(lib, a):
    P = lambda v: None if v is None else v.ctypes.data
    buf = C.create_string_buffer(256)
    nsite = 0 if a["qs"] is None else len(a["qs"])
    st = lib.rism_init_noalloc(C.byref(a["grid"]), C.byref(a["opts"]), a["n"], P(a["xyz"]), P(a["q"]),
                               P(a["sigma"]), P(a["eps"]), a.get("nsite", nsite), P(a["qs"]), P(a["sigs"]),
                               P(a["epss"]), P(a["rho"]), None, None, None, None, None, buf, 256)
    return st, buf.value.decode()


def test_noalloc_rejects_bad_values_before_any_gpu_call(lib):
    """Each bad value is refused by the same checks as the context API, before the GPU is touched (there is
    none here: a call that got past the checks would fail with RISM_E_CUDA instead)."""
    import numpy as np

    from paper_2109_09772_gb300 import rism

    nan = float("nan")
    cases = {
        "nx = 0": dict(grid=rism.GridDesc(0, 8, 8, 0.5, (C.c_double * 3)(0, 0, 0))),
        "nx > 65535": dict(grid=rism.GridDesc(70000, 8, 8, 0.5, (C.c_double * 3)(0, 0, 0))),
        "NaN origin": dict(grid=rism.GridDesc(8, 8, 8, 0.5, (C.c_double * 3)(nan, 0, 0))),
        "h = inf": dict(grid=rism.GridDesc(8, 8, 8, float("inf"), (C.c_double * 3)(0, 0, 0))),
        "kappa = inf": dict(opts=rism.default_options(method=rism.METHOD_DIRECT, kappa=float("inf"))),
        "eta = 0": dict(opts=rism.default_options(method=rism.METHOD_DIRECT, eta=0.0)),
        "lj_rcut NaN": dict(opts=rism.default_options(method=rism.METHOD_DIRECT, lj_rcut=nan)),
        "r_short inf": dict(opts=rism.default_options(method=rism.METHOD_DIRECT, r_short=float("inf"))),
        "NaN in xyz": dict(xyz=np.array([[0.0, nan, 0.0], [1, 1, 1], [2, 2, 2]])),
        "negative sigma": dict(sigma=np.array([2.0, -1.0, 2.0])),
        "negative eps": dict(eps=np.array([0.1, 0.1, -0.1])),
        "Inf charge": dict(q=np.array([1.0, float("inf"), 1.0])),
        "no sites": dict(qs=None, sigs=None, epss=None, nsite=0),
        "negative density": dict(rho=np.array([0.03, -0.06])),
        "NaN solvent sigma": dict(sigs=np.array([nan, 1.0])),
        "too many atoms": dict(n=rism.NOALLOC_MAX_ATOMS + 1, xyz=np.zeros((rism.NOALLOC_MAX_ATOMS + 1, 3)),
                               q=np.zeros(rism.NOALLOC_MAX_ATOMS + 1),
                               sigma=np.ones(rism.NOALLOC_MAX_ATOMS + 1), eps=np.ones(rism.NOALLOC_MAX_ATOMS + 1)),
    }
    for name, over in cases.items():
        st, msg = _call_noalloc(lib, _noalloc_args(rism, **over))
        assert st == rism.E_INVALID, (name, st, msg)
        assert msg, name
    # the treecode is not offered without allocation
    st, _ = _call_noalloc(lib, _noalloc_args(rism, opts=rism.default_options(method=rism.METHOD_TREECODE)))
    assert st == rism.E_UNSUPPORTED


def test_noalloc_rejects_host_outputs_before_any_gpu_call(lib):
    """Outputs are written by kernels: a host pointer is refused (a kernel store there would fault)."""
    import numpy as np

    from paper_2109_09772_gb300 import rism

    a = _noalloc_args(rism)
    host_u = np.zeros((2, 8, 8, 8))
    P = lambda v: v.ctypes.data
    buf = C.create_string_buffer(256)
    st = lib.rism_init_noalloc(C.byref(a["grid"]), C.byref(a["opts"]), a["n"], P(a["xyz"]), P(a["q"]),
                               P(a["sigma"]), P(a["eps"]), 2, P(a["qs"]), P(a["sigs"]), P(a["epss"]), P(a["rho"]),
                               None, P(host_u), None, None, None, buf, 256)
    assert st == rism.E_INVALID
    assert "device memory" in buf.value.decode()
