"""CPU-side checks of the C ABI: the library loads, exports every function
include/wtmd.h declares, and the ctypes mirrors of its structs have the C
layout (offsets compared with a probe compiled by gcc from the header)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wtmd.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def wt():
    import paper_2301_04835_b300 as wt
    from paper_2301_04835_b300 import build

    build.build()
    return wt


def test_library_exports_every_declared_symbol(wt):
    names = _declared()
    assert {"wtmd_create", "cv_define", "step_n", "bias_eval", "fes_grid"} <= set(names)
    lib = wt.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(wt.EXPORTS) == names


def test_struct_layout_matches_header(wt):
    fields = {"wtmd_config": wt.Config, "wtmd_cv_desc": wt.CvDesc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for cname, cls in fields.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "p.c"), os.path.join(d, "p")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-o", exe, src])
        out = subprocess.check_output([exe]).decode().split("\n")
    got = {}
    for l in out:
        if l:
            a, b, c = l.split()
            got[(a, b)] = int(c)
    for cname, cls in fields.items():
        assert got[(cname, "sizeof")] == C.sizeof(cls)
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_create_without_device_fails_cleanly(wt):
    """On a host without a GPU, wtmd_create reports an error instead of
    crashing (there is no CPU fallback)."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a device is present")
    ws = (C.c_int64 * 1)(4)
    c = wt.Config()
    c.precision, c.n_cv = 0, 1
    c.sigma[0], c.w0, c.gamma, c.kT, c.dt, c.mass = 0.1, 1.0, 10.0, 1.0, 1e-3, 1.0
    c.n_walkers, c.walker_size = 1, C.cast(ws, C.POINTER(C.c_int64))
    h = C.c_void_p()
    rc = wt.lib().wtmd_create(C.byref(c), C.byref(h))
    assert rc in (wt.ECUDA, wt.ENOMEM)
    assert not h.value


def test_create_rejects_bad_config_before_touching_the_device(wt):
    ws = (C.c_int64 * 1)(4)
    c = wt.Config()
    c.precision, c.n_cv = 0, 4  # too many CVs
    c.sigma[0], c.w0, c.gamma, c.kT, c.dt, c.mass = 0.1, 1.0, 10.0, 1.0, 1e-3, 1.0
    c.n_walkers, c.walker_size = 1, C.cast(ws, C.POINTER(C.c_int64))
    h = C.c_void_p()
    assert wt.lib().wtmd_create(C.byref(c), C.byref(h)) == wt.EINVAL
    c.n_cv, c.gamma = 1, 0.5  # bias factor must be > 1 (or 0 for standard)
    assert wt.lib().wtmd_create(C.byref(c), C.byref(h)) == wt.EINVAL
