"""CPU-side checks of the C ABI: the library builds, loads, and exports every
function include/perm_f3.h declares (no compute call: no GPU here)."""
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "perm_f3.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("perm_f3", "perm_f3_batch", "perm_f3_range_counts", "perm_f3_counts",
                 "perm_f3_range_counts_async", "perm_f3_batch_async", "pf3_strerror"):
        assert must in names


@pytest.fixture(scope="module")
def libpath():
    from paper_2407_20205_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if " T " in line)
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_reports_errors(libpath):
    from paper_2407_20205_gb300 import binding
    assert binding.version().startswith("perm_f3")
    assert binding.strerror(binding.PF3_EDOMAIN) == "matrix entry outside {0,1,2}"
    assert set(binding.exported_symbols()) <= set(declared_functions())


def test_no_oracle_in_product_path():
    pkg = os.path.join(ROOT, "paper_2407_20205_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "perm_f3_oracle" not in src, f


def test_binding_check_calls_are_well_formed():
    """Every _check(rc, what) call in the binding has exactly two arguments."""
    import ast
    src = open(os.path.join(ROOT, "paper_2407_20205_gb300", "binding.py")).read()
    bad = []
    for node in ast.walk(ast.parse(src)):
        if isinstance(node, ast.Call) and getattr(node.func, "id", None) == "_check":
            if len(node.args) != 2:
                bad.append(node.lineno)
    assert not bad, bad


def test_header_is_c99_and_links(tmp_path, libpath):
    """A C99 program that references every declared function compiles against
    include/perm_f3.h and links with the library (it is not run: no GPU)."""
    names = declared_functions()
    body = "\n".join(f"    p[{k}] = (void (*)(void))&{n};" for k, n in enumerate(names))
    src = tmp_path / "uses_all.c"
    src.write_text(
        '#include "perm_f3.h"\n#include <stdio.h>\n'
        f"int main(void) {{\n    void (*p[{len(names)}])(void);\n{body}\n"
        '    printf("%p\\n", (void*)p[0]);\n    return 0;\n}\n')
    exe = tmp_path / "uses_all"
    libdir = os.path.dirname(libpath)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe), "-L", libdir, "-lperm_f3", f"-Wl,-rpath,{libdir}"], check=True, capture_output=True,
                   text=True)
    assert exe.exists()


def _declarations():
    """(return type, name, [parameter types]) of every function in the header."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    text = "\n".join(l for l in text.splitlines() if not l.strip().startswith("#"))
    text = text.replace('extern "C" {', "")
    out = []
    for stmt in text.split(";"):
        stmt = " ".join(stmt.split())
        if not stmt or stmt.startswith(("typedef", "struct", "}", "extern")) or "{" in stmt:
            stmt = stmt.split("}")[-1].strip() if "}" in stmt else stmt
            if not stmt or stmt.startswith(("typedef", "struct", "extern")):
                continue
        m = re.match(r"^(.*?)\b([a-z][a-z0-9_]*)\s*\((.*)\)$", stmt)
        if not m:
            continue
        ret, name, params = m.group(1).strip(), m.group(2), m.group(3).strip()
        plist = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        types = []
        for p in plist:
            if "*" in p:
                types.append("ptr")
            else:
                types.append(" ".join(p.split()[:-1]).replace("const ", ""))
        out.append(("ptr" if "*" in ret else ret.replace("const ", "").strip(), name, types))
    return out


def test_binding_signatures_match_the_header(libpath):
    """Every function the ctypes layer declares has the header's parameter
    count, pointer/scalar kinds, integer widths and return type: a mismatch
    would pass garbage through the ABI without any error."""
    import ctypes
    from paper_2407_20205_gb300 import binding
    scalar = {"int": ctypes.c_int, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
              "uint64_t": ctypes.c_uint64, "double": ctypes.c_double}
    decl = {name: (ret, types) for ret, name, types in _declarations()}
    assert len(decl) >= 40, sorted(decl)
    checked = 0
    for attr in dir(binding):
        f = getattr(binding, attr)
        name = getattr(f, "__name__", None)
        if not attr.startswith("_lib_") or name not in decl:
            continue
        ret, types = decl[name]
        argtypes = list(f.argtypes or [])
        assert len(argtypes) == len(types), (name, types, argtypes)
        for t, a in zip(types, argtypes):
            if t == "ptr":
                assert a in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(a, "_type_") and \
                    issubclass(a, ctypes._Pointer), (name, t, a)
            else:
                assert ctypes.sizeof(a) == ctypes.sizeof(scalar[t]), (name, t, a)
                if t in ("int", "int32_t", "int64_t"):
                    assert a(-1).value == -1, (name, t, a)   # signed
                if t == "uint64_t":
                    assert a(-1).value > 0, (name, t, a)     # unsigned
                if t == "double":
                    assert a is ctypes.c_double, (name, t, a)
        if ret == "ptr":
            assert f.restype in (ctypes.c_char_p, ctypes.c_void_p), (name, f.restype)
        elif ret == "void":
            assert f.restype is None, (name, f.restype)
        else:
            assert ctypes.sizeof(f.restype) == ctypes.sizeof(scalar[ret]), (name, ret, f.restype)
        checked += 1
    assert checked >= 35, checked


def test_struct_layouts_match_the_binding(tmp_path):
    """sizeof and every field offset of the header's structs, as a C99
    compiler lays them out, equal the ctypes Structures the binding passes."""
    import ctypes
    from paper_2407_20205_gb300 import binding
    structs = {"pf3_config": binding.PF3Config, "pf3_plan_item": binding.PlanItem,
               "pf3_serve_item": binding.ServeItem}
    lines = []
    for cname, cls in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "perm_f3.h"\nint main(void) {\n'
                   + "\n".join(lines) + "\n    return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True, text=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, what, val = line.split()
        got[(cname, what)] = int(val)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, (cname, field)


def test_perm_from_counts_matches_oracle(libpath, oracle):
    """The library's final map of Eq. (2) (a host function: callable without a
    GPU) against the oracle's, on counts up to 2^64 - 1 for every n, and its
    refusal of n outside 0..64."""
    import numpy as np
    from paper_2407_20205_gb300 import binding
    rng = np.random.default_rng(64)
    edges = [0, 1, 2, 3, (1 << 63) - 1, 1 << 63, (1 << 63) + 1, (1 << 64) - 2, (1 << 64) - 1]
    vals = edges + [int(x) for x in rng.integers(0, 1 << 63, 40, dtype=np.uint64)] + \
        [(1 << 63) + int(x) for x in rng.integers(0, 1 << 63, 40, dtype=np.uint64)]
    for n in range(0, 65):
        for k in range(30):
            p = vals[(7 * k + n) % len(vals)]
            m = vals[(11 * k + 3 * n + 1) % len(vals)]
            assert binding.perm_from_counts(n, p, m) == oracle.perm_from_counts(n, p, m), (n, p, m)
    for bad in (-1, 65):
        with pytest.raises(binding.PF3Error):
            binding.perm_from_counts(bad, 1, 0)


def test_no_mod3_arithmetic_in_python_package():
    """The final map lives in the library: the Python package takes something
    mod 3 only where it builds inputs (entries drawn or parsed into {0,1,2},
    pi's digits into F3), never to turn counts into a permanent."""
    import ast
    allowed = {("inputs.py", None), ("pi_matrix.py", "digit_matrix"), ("__main__.py", "read_matrix")}
    pkg = os.path.join(ROOT, "paper_2407_20205_gb300")
    offenders = []
    for f in sorted(os.listdir(pkg)):
        if not f.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(pkg, f)).read())
        for fn in [None] + [x for x in ast.walk(tree) if isinstance(x, ast.FunctionDef)]:
            body = tree if fn is None else fn
            for node in ast.walk(body):
                if (isinstance(node, ast.BinOp) and isinstance(node.op, ast.Mod)
                        and isinstance(node.right, ast.Constant) and node.right.value == 3):
                    owner = None
                    for g in ast.walk(tree):
                        if isinstance(g, ast.FunctionDef) and g.lineno <= node.lineno <= g.end_lineno:
                            owner = g.name
                    if (f, None) not in allowed and (f, owner) not in allowed:
                        offenders.append(f"{f}:{node.lineno}")
    assert not offenders, sorted(set(offenders))


def test_binding_constants_match_the_header():
    """Every #define of the header that the binding mirrors has the same value
    (evaluated by a C compiler, so expressions such as (1 << 24) count)."""
    import re
    from paper_2407_20205_gb300 import binding
    text = open(os.path.join(ROOT, "include", "perm_f3.h")).read()
    names = [m for m in re.findall(r"^#define (PF3_\w+) ", text, re.M)]
    pairs = {}
    for name in names:
        short = name[len("PF3_"):]
        for cand in (name, short):
            if hasattr(binding, cand):
                pairs[name] = getattr(binding, cand)
                break
    # the ones a caller of the binding relies on must be there
    for must in ("PF3_EINVAL", "PF3_ETOOBIG", "PF3_MAX_N", "PF3_CLASS_MAX_COLS", "PF3_NOALLOC_MAX_CTAS",
                 "PF3_LONGRUN_MAX_CHUNK_LOG2", "PF3_VEC_MAX_N", "PF3_TINY_MAX_N"):
        assert must in pairs, must
    import subprocess
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "defs.c")
        with open(src, "w") as f:
            f.write('#include <stdio.h>\n#include "perm_f3.h"\nint main(void) {\n')
            for name in pairs:
                f.write(f'    printf("{name} %lld\\n", (long long)({name}));\n')
            f.write("    return 0;\n}\n")
        exe = os.path.join(d, "defs")
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = dict((k, int(v)) for k, v in (line.split() for line in out.splitlines()))
    for name, val in pairs.items():
        if isinstance(val, int):  # tuples such as SPLIT_CANDIDATES list values, not a count
            assert got[name] == val, (name, got[name], val)
