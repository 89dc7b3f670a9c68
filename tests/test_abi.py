"""The C ABI as a library: it builds, loads without a GPU, exports every
function include/veloxq.h declares, and rejects bad arguments before touching
the device. CPU only: no compute call runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "veloxq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(veloxq_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2501_19221_gb300 import binding
    return binding


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["veloxq_create_dense", "veloxq_create_csr", "veloxq_solve", "veloxq_energy",
                 "veloxq_solve_batch", "veloxq_grad", "veloxq_destroy", "veloxq_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    missing = [n for n in names if not hasattr(lib._lib, n)]
    assert not missing, missing
    assert sorted(lib.EXPORTED) == names


def test_schedule_defaults(lib):
    s = lib.veloxq_schedule_default()
    assert (s.dt, s.a0, s.kappa, s.c0, s.sigma0, s.n_knots, s.readout_every, s.prec, s.path, s.method) == \
        (0.5, 1.0, 1.0, 0.0, pytest.approx(0.1), 0, 50, 0, 0, 0)
    assert s.momentum == pytest.approx(0.9)


def test_struct_layouts_match_the_header(lib, tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C header gives
    (compiled here with the host C compiler)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    structs = {"veloxq_schedule": lib.Schedule, "veloxq_info": lib.Info, "veloxq_timing": lib.Timing}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "veloxq.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_argument_errors_before_device(lib):
    L = lib._lib
    h = ctypes.c_void_p()
    Q = np.eye(2, dtype=np.float32)
    assert L.veloxq_create_dense(None, 2, 2, Q.ctypes.data, None, None) == lib.VELOXQ_EINVAL
    assert L.veloxq_create_dense(ctypes.byref(h), 2, 2, None, None, None) == lib.VELOXQ_EINVAL
    assert L.veloxq_create_dense(ctypes.byref(h), 0, 2, Q.ctypes.data, None, None) == lib.VELOXQ_EINVAL
    assert "n must be >= 1" in lib.veloxq_last_error()
    assert L.veloxq_create_dense(ctypes.byref(h), (1 << 20) + 1, 2, Q.ctypes.data, None, None) == lib.VELOXQ_EINVAL
    assert L.veloxq_create_csr(ctypes.byref(h), 4, None, None, 0, None, None, None) == lib.VELOXQ_EINVAL
    assert L.veloxq_solve(None, 1, 1, None, 0, None, None, None, None) == lib.VELOXQ_EINVAL
    assert L.veloxq_energy(None, 1, None, None, None) == lib.VELOXQ_EINVAL
    assert L.veloxq_grad(None, 1, 1, None, 0, 20, None, None, None, None) == lib.VELOXQ_EINVAL
    L.veloxq_destroy(None)   # no-op


def test_no_device_is_a_cuda_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.VeloxqError) as e:
        lib.veloxq_create_dense(np.eye(3, dtype=np.float32))
    assert e.value.status == lib.VELOXQ_ECUDA
