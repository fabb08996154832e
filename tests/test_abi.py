"""CPU-only checks of the C ABI library: it builds, loads, and exports every
entry point declared in include/ibpme.h (no compute calls without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ibpme.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:ibpme_status|const char\*)\s+(\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2401_04865_gb300 import _build
    try:
        return _build.build()
    except RuntimeError as e:   # nvcc present here; fail loudly if the build breaks
        pytest.fail(str(e))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["pme_setup", "pme_spread", "pme_field", "induced_charge_solve", "body_force_torque",
                 "pme_destroy", "ibpme_bd_step", "ibpme_last_error", "ibpme_get_params", "ibpme_set_stream"]:
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    # nothing else leaks out of the library (internal symbols are hidden)
    extra = [n for n in exported if not (n.startswith("pme_") or n.startswith("ibpme_") or
                                         n in ("induced_charge_solve", "induced_charge_solve_batch",
                                                "body_force_torque"))]
    assert not extra, extra


def test_library_loads_and_binding_matches_header(libpath):
    import paper_2401_04865_gb300 as ib
    lib = ib.load(libpath)
    for n in _declared():
        assert hasattr(lib, n)
        assert n in ib.SIGNATURES
    assert ib.last_error() == ""


def test_struct_layouts_match_header():
    """The ctypes mirrors have the sizes the C compiler gives the header structs."""
    import ctypes
    import tempfile

    import paper_2401_04865_gb300 as ib
    src = r'''
#include <stdio.h>
#include "ibpme.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(ibpme_params), sizeof(ibpme_bodies), sizeof(ibpme_solve_opts),
         sizeof(ibpme_solve_stats), sizeof(ibpme_bd_params));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(v) for v in subprocess.check_output([exe]).split()]
    assert sizes == [ctypes.sizeof(t) for t in (ib.ibpme_params, ib.ibpme_bodies, ib.ibpme_solve_opts,
                                                ib.ibpme_solve_stats, ib.ibpme_bd_params)]
