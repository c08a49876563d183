"""The C-ABI library builds, loads and exports every entry point declared in
include/spock.h; host-only entry points behave (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_01110_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "spock.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(spock_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header(lib):
    from paper_2212_01110_gb300 import spock
    assert set(declared_functions()) == set(spock.EXPORTED)


def test_host_only_calls(lib):
    from paper_2212_01110_gb300 import spock, workloads
    s = spock.spock_default_settings()
    assert s.eps_abs == 1e-6 and s.memory == 3 and s.max_backtracks == 30
    d = workloads.small_binary(0)
    t = spock.spock_tree_create(d["anc"], d["prob"])
    n, N, nl = C.c_int32(), C.c_int32(), C.c_int32()
    assert lib.spock_tree_info(t, C.byref(n), C.byref(N), C.byref(nl)) == 0
    assert (n.value, N.value, nl.value) == (15, 3, 7)
    spock.spock_free(t)
    spock.spock_free(None)
    # absolute probabilities: pi^c must add up to the parent's pi
    pi = np.ones(15)
    for i in range(1, 15):
        pi[i] = pi[d["anc"][i]] * d["prob"][i]
    t = spock.spock_tree_create_abs(d["anc"], pi)
    assert lib.spock_tree_info(t, C.byref(n), C.byref(N), C.byref(nl)) == 0
    assert (n.value, N.value, nl.value) == (15, 3, 7)
    spock.spock_free(t)
    pi[3] *= 2.0
    with pytest.raises(spock.SpockError):
        spock.spock_tree_create_abs(d["anc"], pi)
    pi[3] = -1.0
    with pytest.raises(spock.SpockError):
        spock.spock_tree_create_abs(d["anc"], pi)


@pytest.mark.parametrize("anc,code", [([-1], -1), ([0, 0], -2), ([-1, 0, 0, 1], -2), ([-1, 2, 1], -2),
                                       ([-1, 7], -2)])
def test_bad_tree_codes(lib, anc, code):
    from paper_2212_01110_gb300 import spock
    with pytest.raises(spock.SpockError) as e:
        spock.spock_tree_create(np.array(anc, np.int32), np.ones(len(anc)))
    assert e.value.code == code


def test_bad_probabilities(lib):
    from paper_2212_01110_gb300 import spock
    with pytest.raises(spock.SpockError) as e:
        spock.spock_tree_create(np.array([-1, 0, 0], np.int32), np.array([1.0, 0.3, 0.3]))
    assert e.value.code == -1
    assert "sum to 1" in spock.spock_last_error()


def test_fig1_tree_accepted(lib):
    import json
    from paper_2212_01110_gb300 import spock
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "fig1_tree.json")))
    anc = np.array(g["anc"], np.int32)
    prob = np.ones(len(anc))
    for k, ch in g["children"].items():
        prob[ch] = 1.0 / len(ch)
    t = spock.spock_tree_create(anc, prob)
    n, N, nl = C.c_int32(), C.c_int32(), C.c_int32()
    assert lib.spock_tree_info(t, C.byref(n), C.byref(N), C.byref(nl)) == 0
    assert (n.value, N.value, nl.value) == (9, g["N"], len(g["nonleaf"]))
    spock.spock_free(t)


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures (settings, info, risk measure) have
    the header's field order, offsets and sizes: a C program compiled
    against include/spock.h prints offsetof / sizeof for every field the
    binding declares (a field missing from the header fails to compile)."""
    import json
    import shutil
    import subprocess
    from paper_2212_01110_gb300 import spock
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"spock_settings": spock.Settings, "spock_info": spock.Info, "spock_risk": spock.Risk}
    cname = {"lambda_": "lambda"}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "spock.h"', "int main(void) {", 'printf("{");']
    first = True
    for sname, cls in structs.items():
        for fname, _ in cls._fields_:
            c = cname.get(fname, fname)
            sep = "" if first else ","
            first = False
            lines.append(f'printf("{sep}\\"{sname}.{fname}\\": %zu", offsetof({sname}, {c}));')
        lines.append(f'printf(",\\"{sname}.sizeof\\": %zu", sizeof({sname}));')
    lines += ['printf("}\\n");', "return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = json.loads(subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout)
    for sname, cls in structs.items():
        for fname, _ in cls._fields_:
            assert got[f"{sname}.{fname}"] == getattr(cls, fname).offset, (sname, fname)
        assert got[f"{sname}.sizeof"] == C.sizeof(cls), sname


def _header_prototypes():
    src = open(os.path.join(ROOT, "include", "spock.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"^\s*(int|void|const char\*)\s+(spock_\w+)\s*\(([^;]*?)\)\s*;", src, flags=re.M | re.S):
        args = [a.strip() for a in m.group(3).replace("\n", " ").split(",") if a.strip() and a.strip() != "void"]
        out[m.group(2)] = (m.group(1), args)
    return out


def _c_kind(arg):
    if "*" in arg:
        return "ptr"
    typ = " ".join(arg.split()[:-1]).replace("const ", "")
    return {"int32_t": "i32", "int": "i32", "int64_t": "i64", "double": "f64"}[typ]


def _py_kind(t):
    if t in (C.c_int32, C.c_int):
        return "i32"
    if t is C.c_int64:
        return "i64"
    if t is C.c_double:
        return "f64"
    return "ptr"


def test_binding_signatures_match_the_header():
    """Every function's argument count and the kind of each argument (32-bit
    integer, 64-bit integer, double or pointer) and its return type agree
    between include/spock.h and the binding's ctypes declarations."""
    from paper_2212_01110_gb300 import spock
    protos = _header_prototypes()
    assert set(protos) == set(spock._sig)
    for name, (ret, args) in protos.items():
        pargs, pres = spock._sig[name]
        assert [_c_kind(a) for a in args] == [_py_kind(t) for t in pargs], name
        want = {"int": C.c_int, "void": None, "const char*": C.c_char_p}[ret]
        assert pres is want, name


def test_risk_marshalling():
    """spock_risk entries built by the binding carry each node's sizes and
    point at row-major copies of b, E and F that stay alive with the array
    (leaves: zeroed entries)."""
    from paper_2212_01110_gb300 import spock, workloads
    d = workloads.risk_measures(workloads.small_binary(1, a=0.5), "tv", radius=0.3)
    arr, keep = spock._risk_array(d["risk"])
    assert len(arr) == len(d["risk"])
    for i, r in enumerate(d["risk"]):
        e = arr[i]
        if r is None:
            assert e.ny == 0 and not e.b
            continue
        b, E = np.asarray(r["b"], float), np.asarray(r["E"], float)
        F = np.asarray(r.get("F", np.zeros((b.size, 0))), float)
        assert (e.ny, e.n_nu, e.kp) == (b.size, F.shape[1] if F.ndim == 2 else 0, int(r["kp"]))
        np.testing.assert_array_equal(np.ctypeslib.as_array(e.b, (b.size,)), b)
        np.testing.assert_array_equal(np.ctypeslib.as_array(e.E, (E.size,)), E.ravel())
        if e.n_nu:
            np.testing.assert_array_equal(np.ctypeslib.as_array(e.F, (F.size,)), F.ravel())
    assert keep


def test_binding_fails_loudly_without_the_library(tmp_path):
    """A copy of the binding next to no built library raises ImportError on
    import: there is no CPU fallback."""
    import importlib.util
    import shutil
    pkg = tmp_path / "pkg"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_2212_01110_gb300", "spock.py"), pkg / "spock.py")
    spec = importlib.util.spec_from_file_location("spock_copy", pkg / "spock.py")
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)


def test_status_codes_match_the_header():
    from paper_2212_01110_gb300 import spock
    src = open(os.path.join(ROOT, "include", "spock.h")).read()
    for name, val in re.findall(r"\b(SPOCK_(?:OK|MAX_ITER|ERR_\w+|FP64|FP32))\s*=\s*(-?\d+)", src):
        assert getattr(spock, name) == int(val), name
    assert re.search(r"#define SPOCK_DENSE_COST (\d+)", src).group(1) == str(spock.SPOCK_DENSE_COST)


def test_product_path_does_not_use_the_oracle():
    """No module of the package imports, loads or runs anything under
    oracle/ (the oracle is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2212_01110_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", src, flags=re.M), f
                assert "riccati_cpu" not in src and "oracle/" not in src, f


def test_oracle_uses_only_the_input_generators():
    """The oracle imports nothing of the package but the seeded input
    generators (workloads.py), which themselves hold no arithmetic of the
    method: they import numpy only."""
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        if f.endswith((".py", ".cpp")):
            src = open(os.path.join(odir, f)).read()
            for mod in re.findall(r"paper_2212_01110_gb300(?:\.(\w+)|\s+import\s+(\w+))", src):
                assert "workloads" in mod, (f, mod)
            assert "libspock" not in src and "csrc" not in src, f
    wl = open(os.path.join(ROOT, "paper_2212_01110_gb300", "workloads.py")).read()
    imports = set(re.findall(r"^\s*(?:from\s+(\S+)\s+import|import\s+(\S+))", wl, flags=re.M))
    assert {m for pair in imports for m in pair if m} <= {"__future__", "numpy"}
