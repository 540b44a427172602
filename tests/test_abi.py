"""The C ABI builds, loads and exports every symbol include/*.h declares,
and the Python structure mirrors the C layout (CPU only: no compute call)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"NBODY_API\s+[\w\s\*]+?\b(nbody_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2511_22468_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("nbody_create", "nbody_step", "nbody_integrate", "nbody_vjp",
                     "nbody_destroy", "nbody_set_state", "nbody_energy",
                     "nbody_get_status", "nbody_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (nbody_\w+)", out))
    assert exported == set(declared_symbols())


def test_binding_lists_the_same_names(libpath):
    from paper_2511_22468_gb300 import nbody
    assert set(nbody.EXPORTED) == set(declared_symbols())
    for name in declared_symbols():
        assert callable(getattr(nbody, name))


def test_strerror_and_counter_are_host_only(libpath):
    from paper_2511_22468_gb300 import nbody
    assert nbody.nbody_strerror(0) == "ok"
    assert "tape" in nbody.nbody_strerror(nbody.NBODY_ESTATE)
    assert nbody.nbody_strerror(-99) == "unknown status"
    assert nbody.nbody_launch_count() >= 0


def test_params_struct_layout_matches_c(tmp_path, libpath):
    from paper_2511_22468_gb300 import nbody
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "nbody.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(nbody_params),
         offsetof(nbody_params, checkpoint_every), offsetof(nbody_params, tape_mode),
         offsetof(nbody_params, nfw_M), offsetof(nbody_params, center),
         offsetof(nbody_params, center_vel));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    vals = [int(t) for t in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    P = nbody.nbody_params
    assert vals == [ctypes.sizeof(P), P.checkpoint_every.offset, P.tape_mode.offset,
                    P.nfw_M.offset, P.center.offset, P.center_vel.offset]


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_2511_22468_gb300 import nbody
    monkeypatch.setattr(nbody, "_lib", None)
    monkeypatch.setattr(nbody, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        nbody.lib()


def test_empty_and_invalid_inputs_are_refused_before_any_device_work(libpath):
    """Empty systems (n = 0), an empty batch member, a zero softening and
    NULL outputs return NBODY_EINVAL from the argument checks, which come
    before any device query or allocation (so this runs without a GPU)."""
    from paper_2511_22468_gb300 import nbody
    lib = nbody.lib()
    p = nbody.make_params(1.0, 0.01, 1e-3)
    h = ctypes.c_void_p()
    assert lib.nbody_create(ctypes.byref(h), 0, ctypes.byref(p), None) == nbody.NBODY_EINVAL
    assert lib.nbody_create(ctypes.byref(h), -5, ctypes.byref(p), None) == nbody.NBODY_EINVAL
    assert not h.value
    p0 = nbody.make_params(1.0, 0.0, 1e-3)           # eps = 0: the GPU path needs eps > 0
    assert lib.nbody_create(ctypes.byref(h), 10, ctypes.byref(p0), None) == nbody.NBODY_EINVAL
    offs = (ctypes.c_int64 * 3)(0, 5, 5)            # second member empty
    ps = (nbody.nbody_params * 2)(p, p)
    assert lib.nbody_create_batch(ctypes.byref(h), 2, offs, ps, None) == nbody.NBODY_EINVAL
    offs = (ctypes.c_int64 * 2)(1, 5)                # offsets must start at 0
    assert lib.nbody_create_batch(ctypes.byref(h), 1, offs, ps, None) == nbody.NBODY_EINVAL
    cen = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    buf = (ctypes.c_double * 3)()
    assert lib.nbody_pair_accel(0, buf, buf, ctypes.c_double(1.0), ctypes.c_double(0.01), cen,
                                buf, None) == nbody.NBODY_EINVAL
    assert lib.nbody_pair_accel(1, buf, buf, ctypes.c_double(1.0), ctypes.c_double(0.01), cen,
                                None, None) == nbody.NBODY_EINVAL
