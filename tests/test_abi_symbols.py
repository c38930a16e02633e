"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/*.h declares (no compute calls on CPU)."""

import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(nmf_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_declared_symbols():
    from paper_1904_07935_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared_functions()
    assert {"nmf_init", "nmf_iterate", "nmf_error", "nmf_destroy"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_1904_07935_b300 import nmf
    assert nmf.lib.nmf_status_str(nmf.NMF_ETIMEOUT) == b"device wait timed out"
    assert nmf.lib.nmf_status_str(99) == b"unknown status"


def test_null_arguments_rejected_without_gpu():
    from paper_1904_07935_b300 import nmf
    assert nmf.lib.nmf_init(None, None) == nmf.NMF_EINVAL
    assert nmf.lib.nmf_iterate(None, 1) == nmf.NMF_EINVAL
    assert nmf.lib.nmf_error(None, None, None) == nmf.NMF_EINVAL
    p = nmf.Problem()
    p.V, p.D, p.K = 10, 8, 9            # K > min(V, D)
    h = ctypes.c_void_p()
    assert nmf.lib.nmf_init(ctypes.byref(p), ctypes.byref(h)) == nmf.NMF_EINVAL
    p.K = 0
    assert nmf.lib.nmf_init(ctypes.byref(p), ctypes.byref(h)) == nmf.NMF_EINVAL
