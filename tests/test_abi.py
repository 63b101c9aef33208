"""CPU tests of the C-ABI library: it loads without a GPU, exports every
function include/*.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


@pytest.fixture(scope="module")
def csl():
    import __graft_entry__ as g
    g.build()
    import paper_2408_00488_gb300 as csl
    return csl


def declared_functions():
    text = "\n".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s*(csl_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("csl_plan_create", "csl_plan_destroy", "csl_precondition", "csl_apply", "csl_solve",
                     "csl_solve_host", "csl_adjoint", "csl_coef_grad", "csl_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(csl):
    lib = ctypes.CDLL(csl._binding.LIBPATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(csl):
    assert csl.version().startswith("csl")
    for code, name in enumerate(["CSL_OK", "CSL_INVALID_ARG", "CSL_UNSUPPORTED_SIZE", "CSL_SINGULAR_PRECOND",
                                 "CSL_BREAKDOWN", "CSL_NOT_CONVERGED", "CSL_TIMEOUT", "CSL_CUDA_ERROR",
                                 "CSL_OUT_OF_MEMORY"]):
        assert csl.status_string(code) == name
    assert csl.status_string(99) == "CSL_UNKNOWN_STATUS"


def test_options_init(csl):
    b = csl._binding
    o = b.PlanOptions()
    assert csl.lib.csl_plan_options_init(ctypes.byref(o)) == 0
    assert o.precision == 0 and o.use_graph == 1 and o.lines_per_cta == 0 and o.autotune == 1
    assert o.gamma_override != o.gamma_override  # NaN: derive gamma from the samples
    assert csl.lib.csl_plan_options_init(None) == b.INVALID_ARG


def _create(csl, dim, n, ptrs, alpha=1.0, beta=1.0):
    b = csl._binding
    h = ctypes.c_void_p()
    nn = (ctypes.c_int64 * 3)(*n)
    pp = (ctypes.c_void_p * 3)(*ptrs)
    return csl.lib.csl_plan_create(ctypes.byref(h), dim, nn, pp, alpha, beta, None, None), h


def test_host_side_argument_validation(csl):
    b = csl._binding
    fake = 0x1000  # never dereferenced: validation fails first
    assert _create(csl, 4, (7, 7, 7), (fake, fake, fake))[0] == b.INVALID_ARG
    assert _create(csl, 2, (7, 7, 1), (fake, None, None))[0] == b.INVALID_ARG
    assert _create(csl, 2, (0, 7, 1), (fake, fake, None))[0] == b.INVALID_ARG
    assert _create(csl, 2, (8, 7, 1), (fake, fake, None))[0] == b.UNSUPPORTED_SIZE
    # 2D lines up to 16384 points in FP64 (4096 in the FP32 forms), 3D up to 1024
    assert _create(csl, 2, (32767, 7, 1), (fake, fake, None))[0] == b.UNSUPPORTED_SIZE
    assert _create(csl, 3, (2047, 7, 7), (fake, fake, fake))[0] == b.UNSUPPORTED_SIZE
    assert _create(csl, 3, (7, 7, 2), (fake, fake, fake))[0] == b.UNSUPPORTED_SIZE
    assert _create(csl, 2, (7, 7, 1), (fake, fake, None), alpha=float("nan"))[0] == b.INVALID_ARG
    assert _create(csl, 2, (7, 7, 1), (fake, fake, None), beta=float("inf"))[0] == b.INVALID_ARG
    for fn in ("csl_solve", "csl_adjoint", "csl_solve_host"):
        assert getattr(csl.lib, fn)(None, None, None, 1e-8, 10, None) == b.INVALID_ARG
    assert csl.lib.csl_apply(None, None, None) == b.INVALID_ARG
    assert csl.lib.csl_precondition(None, None, None) == b.INVALID_ARG
    assert csl.lib.csl_coef_grad(None, None, None, None) == b.INVALID_ARG
    assert csl.lib.csl_plan_workspace_bytes(None) == 0
    assert csl.lib.csl_plan_config(None) == b""
    csl.lib.csl_plan_destroy(None)


C_TYPES = {"int": ctypes.c_int, "double": ctypes.c_double, "int64_t": ctypes.c_int64,
           "const double*": ctypes.c_void_p, "double*": ctypes.c_void_p, "void*": ctypes.c_void_p}


def header_struct(name):
    """(field name, ctypes type, array length) of `typedef struct name {...} name;` in csl.h."""
    text = open(os.path.join(ROOT, "include", "csl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), text, flags=re.S).group(1)
    out = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        m = re.match(r"(const\s+)?(\w+)\s*(\*?)\s*(.*)$", decl)
        assert m, decl
        ctype = ((m.group(1) or "") + m.group(2) + m.group(3)).strip()
        for name in m.group(4).split(","):  # a declaration may list several fields
            d = re.match(r"\s*(\w+)\s*(?:\[(\d+)\])?\s*$", name)
            assert d, decl
            out.append((d.group(1), C_TYPES[ctype], int(d.group(2) or 1)))
    return out


@pytest.mark.parametrize("cname,pyname", [("csl_plan_options", "PlanOptions"), ("csl_solve_info", "SolveInfo"),
                                          ("csl_system_desc", "SystemDesc"), ("csl_paradiag_info", "ParaDiagInfo"),
                                          ("csl_helmholtz_info", "HelmholtzInfo")])
def test_binding_structs_match_the_header(csl, cname, pyname):
    """The ctypes mirrors carry the header's fields in order, with the same
    types and array lengths, so the struct sizes and offsets agree."""
    py = getattr(csl._binding, pyname)
    got = []
    for fname, ftype in py._fields_:
        n = getattr(ftype, "_length_", 1)
        base = getattr(ftype, "_type_", ftype) if n > 1 or hasattr(ftype, "_length_") else ftype
        got.append((fname, base, n))
    want = header_struct(cname)
    assert [(f, n) for f, _, n in got] == [(f, n) for f, _, n in want]
    for (f, t_got, _), (_, t_want, _) in zip(got, want):
        assert ctypes.sizeof(t_got) == ctypes.sizeof(t_want), (cname, f)


def test_options_init_enables_the_fast_paths(csl):
    o = csl._binding.PlanOptions()
    assert csl.lib.csl_plan_options_init(ctypes.byref(o)) == 0
    assert o.programmatic_launch == 1 and o.float_pair_stencil == 1
    assert o.update_mode == 0 and o.body_iters == 0 and o.warm_start == 0 and o.history == 0
    assert all(r == 0 for r in o.reserved)


def test_tune_cache_files_checked_on_the_host(csl, tmp_path):
    """The tuner's cache file is written and read on the host: a malformed
    file loads nothing, and a missing one is an argument error."""
    b = csl._binding
    good = tmp_path / "tc.txt"
    assert csl.lib.csl_tune_cache_save(str(good).encode()) == b.OK
    assert open(good).read().splitlines()[0] == "csl-tune-cache 1"
    assert csl.lib.csl_tune_cache_load(str(good).encode()) == b.OK
    for body in ("not a cache\n", "csl-tune-cache 1\n4 2 1000 7 1 0 4\n", "csl-tune-cache 1\n4 2 1024 7 1 5 4\n",
                 "csl-tune-cache 1\n4 2 1024 7 1 0 3\n", "csl-tune-cache 1\n4 2 1024\n"):
        bad = tmp_path / "bad.txt"
        bad.write_text(body)
        assert csl.lib.csl_tune_cache_load(str(bad).encode()) == b.INVALID_ARG, body
    assert csl.lib.csl_tune_cache_load(str(tmp_path / "missing.txt").encode()) == b.INVALID_ARG
    assert csl.lib.csl_tune_cache_load(None) == b.INVALID_ARG
    assert csl.lib.csl_solve_history(None, None, 0, None) == b.INVALID_ARG
