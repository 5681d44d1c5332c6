"""The C-ABI library builds, loads and exports every entry point that
include/fgx.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2208_00001_gb300 import build
    return build.build()


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(fgx_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    for n in ["fgx_geodesic2d", "fgx_geodesic3d", "fgx_geodesic_batched",
              "fgx_geodesic2d_fwd_train", "fgx_geodesic2d_bwd", "fgx_geodesic3d_bwd"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(libpath):
    lib = ctypes.CDLL(libpath)
    lib.fgx_status_string.restype = ctypes.c_char_p
    assert lib.fgx_status_string(0) == b"ok"
    assert lib.fgx_status_string(-6) == b"device wait timed out"
    assert lib.fgx_status_string(12345) == b"unknown status"
    assert lib.fgx_version() >= 100


def test_binding_refuses_cpu_tensors(libpath):
    import torch
    import paper_2208_00001_gb300 as fgx
    x = torch.zeros(1, 1, 4, 4)
    with pytest.raises(ValueError, match="CUDA"):
        fgx.geodesic2d(x, x, 1.0, 0.5, 1)


def test_size_queries_without_device_do_not_crash(libpath):
    """Without a usable sm_103 device every planning call answers with a
    status code (no CPU fallback, no crash)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    lib = ctypes.CDLL(libpath)
    n = ctypes.c_size_t(0)
    st = lib.fgx_geodesic_workspace_size(2, ctypes.c_int64(1), ctypes.c_int64(1),
                                         ctypes.c_int64(1), ctypes.c_int64(8), ctypes.c_int64(8),
                                         None, ctypes.byref(n))
    assert st == -7  # FGX_ERR_DEVICE


def test_header_compiles_as_c(tmp_path):
    """include/fgx.h is plain C (C99): a C caller can include it and take the
    address of every declared entry point."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = _declared()
    src = tmp_path / "use_fgx.c"
    src.write_text('#include "fgx.h"\n'
                   "typedef void (*entry)(void);\n"
                   "entry entry_points[] = {\n" +
                   "".join(f"    (entry){n},\n" for n in names) +
                   "};\nint main(void) { return entry_points[0] == 0; }\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("cname,pyname", [("fgx_options", "Options"),
                                          ("fgx_instance", "Instance"),
                                          ("fgx_batched_plan", "BatchedPlanC")])
def test_binding_structs_match_the_header(tmp_path, cname, pyname):
    """The binding's ctypes mirrors of the header's structs have the C sizes
    and field offsets (compiled with the host C compiler)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import paper_2208_00001_gb300 as fgx
    py = getattr(fgx, pyname)
    fields = [f[0] for f in py._fields_]
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "fgx.h"\n'
                   "int main(void) {\n"
                   f'    printf("%zu\\n", sizeof({cname}));\n' +
                   "".join(f'    printf("%zu\\n", offsetof({cname}, {f.rstrip("_")}));\n'
                           for f in fields) +  # lambda_ mirrors the C field lambda
                   "    return 0;\n}\n")
    exe = tmp_path / "sizes"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True,
                                          text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(py), (cname, out[0], ctypes.sizeof(py))
    for f, off in zip(fields, out[1:]):
        assert getattr(py, f).offset == off, (cname, f)


def test_no_gpu_reports_no_device(libpath):
    """Without a usable GPU the library answers FGX_ERR_DEVICE (no CPU path,
    no crash) and the binding raises."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = ctypes.CDLL(libpath)
    f = lib.fgx_geodesic_workspace_size
    f.argtypes = [ctypes.c_int32] + [ctypes.c_int64] * 5 + [ctypes.c_void_p,
                                                           ctypes.POINTER(ctypes.c_size_t)]
    f.restype = ctypes.c_int32
    n = ctypes.c_size_t(0)
    assert f(2, 1, 1, 1, 64, 64, None, ctypes.byref(n)) == -7  # FGX_ERR_DEVICE
    import paper_2208_00001_gb300 as fgx
    with pytest.raises(fgx.FgxError):
        fgx.workspace_size(2, 1, 1, 1, 64, 64)
    with pytest.raises(ValueError):
        fgx.geodesic2d(torch.zeros(1, 1, 8, 8), torch.zeros(1, 1, 8, 8), 1.0, 0.5, 1)
