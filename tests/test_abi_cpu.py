"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every function include/lqcd.h declares."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "lqcd.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(lqcd_[a-z0-9_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    lib = __graft_entry__._load_builder().build()
    names = _declared()
    assert "lqcd_dslash" in names and "lqcd_solve" in names and len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lqcd_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    dll = ctypes.CDLL(lib)
    for n in names:
        getattr(dll, n)


def test_binding_reports_errors_without_gpu():
    import paper_2001_05706_gb300 as L
    try:
        import torch
        if torch.cuda.is_available():
            return
    except ImportError:
        pass
    try:
        L.lqcd_create((4, 4, 4, 4))
    except L.LqcdError as e:
        assert e.status in (L.LQCD_ERR_OOM, L.LQCD_ERR_CUDA)
    else:
        raise AssertionError("context creation succeeded without a GPU")
    try:
        L.lqcd_create((4, 3, 4, 4))
    except L.LqcdError as e:
        assert e.status == L.LQCD_ERR_ARG and "even" in str(e)


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the parameter and info structs match the C
    compiler's layout (sizes and the offset of every field)."""
    import paper_2001_05706_gb300 as L
    structs = {"lqcd_solve_params": L.lqcd_solve_params, "lqcd_solve_info": L.lqcd_solve_info,
               "lqcd_overlap_params": L.lqcd_overlap_params, "lqcd_overlap_info": L.lqcd_overlap_info,
               "lqcd_overlap_eigen_params": L.lqcd_overlap_eigen_params,
               "lqcd_overlap_eigen_info": L.lqcd_overlap_eigen_info}
    lines, expect = [], []
    for cname, py in structs.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(py))
        for fname, _ in py._fields_:
            cfield = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("%zu\\n", offsetof({cname}, {cfield}));')
            expect.append(getattr(py, fname).offset)
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lqcd.h"\nint main(void){' + "".join(lines) +
                   ' return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == expect


def test_enum_values_match_header(tmp_path):
    """Every enum constant the binding defines has the header's value."""
    import paper_2001_05706_gb300 as L
    names = [n for n in dir(L) if n.startswith("LQCD_") and isinstance(getattr(L, n), int)]
    assert len(names) >= 40
    lines = "".join(f'printf("%d\\n", (int){n});' for n in names)
    src = tmp_path / "en.c"
    src.write_text('#include <stdio.h>\n#include "lqcd.h"\nint main(void){' + lines + ' return 0;}\n')
    exe = tmp_path / "en"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == [getattr(L, n) for n in names], names


def test_multigrid_entry_points_refuse_a_null_context():
    """Every lqcd_mg_* call checks its context before any CUDA call."""
    import ctypes
    import paper_2001_05706_gb300 as L
    d = (ctypes.c_int * 4)(4, 4, 4, 4)
    p = ctypes.c_void_p(16)
    two = (ctypes.c_double * 2)(1.0, 0.0)
    calls = {
        "lqcd_mg_fine_stencil": (None, p, p, p),
        "lqcd_mg_apply": (None, d, 12, p, p, p, p, p),
        "lqcd_mg_orthonormalize": (None, d, 12, d, 4, p, p),
        "lqcd_mg_prolong": (None, d, 12, d, 8, p, p, p),
        "lqcd_mg_restrict": (None, d, 12, d, 8, p, p, p),
        "lqcd_mg_coarsen": (None, d, 12, d, 8, p, p, p, p, p, p, p),
        "lqcd_mg_dots": (None, 16, 1, p, p, (ctypes.c_double * 2)()),
        "lqcd_mg_axpys": (None, 16, 1, two, p, p),
        "lqcd_mg_axpby": (None, 16, two, p, two, p),
    }
    for name, args in calls.items():
        assert getattr(L._lib, name)(*args) == L.LQCD_ERR_ARG, name
        assert b"context" in L._lib.lqcd_last_error(), name
