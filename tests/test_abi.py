"""The C-ABI library loads, exports every function include/gofd.h declares,
and rejects bad host inputs before touching the device (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gofd.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gofd_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_14437_gb300 import _native, build_native
    if not os.path.exists(_native.LIB_PATH):
        build_native.build()
    return _native.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gofd_build", "gofd_apply", "gofd_solve", "gofd_destroy", "gofd_last_error",
                 "gofd_export_transfer", "gofd_get_coefficients"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2307_14437_gb300 import _native
    assert set(_declared()) == set(_native.EXPORTS)


def _build(lib, d, verts, simp, alpha, h, lo, hi):
    from paper_2307_14437_gb300 import _native as N
    v = np.ascontiguousarray(verts, dtype=np.float64)
    s = np.ascontiguousarray(simp, dtype=np.int32)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    out = C.c_void_p()
    st = lib.gofd_build(d, v.ctypes.data, len(v), s.ctypes.data, len(s), alpha, h, lo.ctypes.data,
                        hi.ctypes.data, None, C.byref(out))
    return N.STATUS[st], lib.gofd_last_error(None).decode()


TRI = (np.array([[0.0, 0.0], [0.5, 0.0], [0.0, 0.5]]), np.array([[0, 1, 2]]))


def test_host_validation_rejects_bad_dimension(lib):
    st, msg = _build(lib, 4, np.zeros((5, 4)), np.zeros((1, 5)), 1.0, 0.5, [-1] * 4, [1] * 4)
    assert st == "GOFD_E_ARG" and "d must be" in msg


def test_host_validation_rejects_bad_alpha(lib):
    st, _ = _build(lib, 2, *TRI, 2.5, 0.5, [-1, -1], [1, 1])
    assert st == "GOFD_E_ARG"


def test_host_validation_rejects_non_integral_grid(lib):
    st, msg = _build(lib, 2, *TRI, 1.0, 0.3, [-1, -1], [1, 1])
    assert st == "GOFD_E_GRID"


def test_host_validation_rejects_vertex_outside_box(lib):
    v = TRI[0].copy()
    v[1, 0] = 1.5
    st, _ = _build(lib, 2, v, TRI[1], 1.0, 0.5, [-1, -1], [1, 1])
    assert st == "GOFD_E_OUTSIDE_BOX"


def test_host_validation_rejects_bad_index(lib):
    st, _ = _build(lib, 2, TRI[0], np.array([[0, 1, 3]]), 1.0, 0.5, [-1, -1], [1, 1])
    assert st == "GOFD_E_ARG"


def test_host_validation_rejects_too_few_grid_nodes(lib):
    # Remark 3.2: (2N+1)^d >= N_v is needed for full column rank
    import meshgen as mg
    v, s = mg.disk_ring_mesh(rings=6, seed=1)
    st, _ = _build(lib, 2, v, s, 1.0, 0.5, [-1, -1], [1, 1])
    assert st == "GOFD_E_TOO_FEW_GRID_NODES"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2307_14437_gb300 import _native
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "libgofd.so"))
    with pytest.raises(ImportError):
        _native.load()


def _header_fields(struct_name):
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + struct_name + r"\s*;", src).group(1)
    names = []
    for decl in filter(None, (d.strip() for d in body.split(";"))):
        parts = re.sub(r"\[\s*\d+\s*\]", "", decl).split(",")   # "int64_t n_v, n_e", "int n[3]"
        names.append(parts[0].split()[-1])
        names += [q.strip() for q in parts[1:]]
    return names


def test_binding_structs_match_the_header(tmp_path):
    # the ctypes mirrors of the ABI's structs: same fields in the same order,
    # same offsets and size as the C compiler lays out include/gofd.h
    import shutil
    import subprocess
    from paper_2307_14437_gb300 import _native as N
    gcc = shutil.which("gcc") or shutil.which("cc")
    if not gcc:
        pytest.skip("no C compiler")
    structs = {"gofd_options": N.Options, "gofd_solve_info": N.SolveInfo, "gofd_info": N.Info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gofd.h"', "int main(void) {"]
    for cname, cls in structs.items():
        assert [f for f, _ in cls._fields_] == _header_fields(cname), cname
        lines.append(f'printf("{cname} . %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for row in filter(None, out):
        cname, field, value = row.split()
        cls = structs[cname]
        want = C.sizeof(cls) if field == "." else getattr(cls, field).offset
        assert int(value) == want, (cname, field, int(value), want)
