"""The C-ABI library loads and exports every entry point of include/l1ls.h (no GPU needed),
and the ctypes structures of the binding match the C layout compiled by gcc."""

import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "l1ls.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(l1ls_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["l1ls_generate", "l1ls_matvec", "l1ls_rmatvec", "l1ls_solve_fista", "l1ls_solve_pdncg",
                     "l1ls_create", "l1ls_destroy", "l1ls_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1503_03520_gb300 as l1
    lib = ctypes.CDLL(l1.library_path)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_header():
    import paper_1503_03520_gb300 as l1
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "l1ls.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(l1ls_gen_params), sizeof(l1ls_inst_info), sizeof(l1ls_solve_opts),
         sizeof(l1ls_result));
  printf("%zu %zu %zu\n", offsetof(l1ls_gen_params, right_stages), offsetof(l1ls_solve_opts, ls_max),
         offsetof(l1ls_result, status));
  printf("%zu %zu %zu %zu\n", offsetof(l1ls_gen_params, gamma), offsetof(l1ls_solve_opts, f_target),
         offsetof(l1ls_result, L), offsetof(l1ls_inst_info, device_bytes));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    sizes = [int(v) for v in out]
    assert sizes[:4] == [ctypes.sizeof(l1.GenParams), ctypes.sizeof(l1.InstInfo), ctypes.sizeof(l1.SolveOpts),
                         ctypes.sizeof(l1.Result)]
    assert sizes[4] == l1.GenParams.right_stages.offset
    assert sizes[5] == l1.SolveOpts.ls_max.offset
    assert sizes[6] == l1.Result.status.offset
    assert sizes[7:] == [l1.GenParams.gamma.offset, l1.SolveOpts.f_target.offset, l1.Result.L.offset,
                         l1.InstInfo.device_bytes.offset]


def test_defaults_without_gpu():
    import paper_1503_03520_gb300 as l1
    p = l1.gen_params({"m": 64, "n": 32, "value_dtype": "f32"})
    assert p.m == 64 and p.n == 32 and p.value_dtype == 1 and p.right_stages == 1 and p.left_stages == 1
    o = l1.solve_opts(tol=1e-8)
    assert o.rel_gap_tol == 1e-8 and o.mu == 1e-5 and o.ls_max == 50 and o.pcg_rtol == 0.1
    assert o.f_target == float("-inf") and o.restart == 0 and o.accum == 0
    q = l1.gen_params({})
    assert q.gamma == 100.0 and q.xstar_mode == 0 and q.sigma_mode == 0 and q.matrix_free == 0


def test_footprint_is_monotone_without_gpu():
    """The serving admission estimate (host arithmetic only): larger instances, more stages,
    wider values and pdNCG's larger work space never lower it."""
    import paper_1503_03520_gb300 as l1
    base = {"m": 4096, "n": 2048, "right_stages": 2, "value_dtype": "f32"}
    f0 = l1.footprint(base)
    assert f0 > 0
    assert l1.footprint(dict(base, m=8192, n=4096)) > f0
    assert l1.footprint(dict(base, right_stages=4)) > f0
    assert l1.footprint(dict(base, value_dtype="f64")) > f0
    assert l1.footprint(base, "pdncg") >= f0


def test_create_fails_cleanly_without_device():
    import torch
    import paper_1503_03520_gb300 as l1
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(l1.L1LSError):
        l1.Context(0)


def test_binding_refuses_to_import_without_the_library():
    """No fallback: a copy of the binding next to no libl1ls.so raises ImportError on import."""
    import sys
    src = os.path.join(ROOT, "paper_1503_03520_gb300", "__init__.py")
    with tempfile.TemporaryDirectory() as d:
        pkg = os.path.join(d, "l1ls_nolib")
        os.makedirs(pkg)
        with open(src) as f, open(os.path.join(pkg, "__init__.py"), "w") as g:
            g.write(f.read())
        r = subprocess.run([sys.executable, "-c", "import l1ls_nolib"], cwd=d, capture_output=True, text=True)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libl1ls.so is not built" in r.stderr


def test_product_sources_do_not_reach_the_oracle():
    """The package (binding, build script, CUDA sources) never names the oracle package."""
    pkg = os.path.join(ROOT, "paper_1503_03520_gb300")
    hits = []
    for dirpath, _dirs, files in os.walk(pkg):
        for name in files:
            if name.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, name)).read()
                if re.search(r"\boracle\b", text):
                    hits.append(name)
    assert not hits, hits


def _prototypes():
    """name -> (return type, [parameter types]) for every function prototype in the header."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    out = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w \t]*?\**)\s*\b(l1ls_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text):
        ps = [p.strip() for p in " ".join(params.split()).split(",") if p.strip()]
        if ps == ["void"]:
            ps = []
        types = []
        for p in ps:
            p = re.sub(r"\bconst\b", "", p)
            m = re.match(r"(.*?)([A-Za-z_]\w*)$", p.strip())       # drop the parameter name
            t = (m.group(1) if m and ("*" in m.group(1) or m.group(1).strip()) else p)
            types.append(" ".join(t.replace("*", " * ").split()))
        out[name] = (" ".join(re.sub(r"\bconst\b", "", ret).replace("*", " * ").split()), types)
    return out


def test_binding_signatures_match_header_prototypes():
    """Every header prototype has a ctypes signature in the binding with the same arity and the
    same scalar widths, and every pointer parameter is a pointer on the Python side."""
    import paper_1503_03520_gb300 as l1
    scalars = {"double": ctypes.c_double, "int": ctypes.c_int, "int32_t": ctypes.c_int32,
               "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64, "uint32_t": ctypes.c_uint32,
               "size_t": ctypes.c_size_t, "l1ls_dtype": ctypes.c_int, "l1ls_status": ctypes.c_int}
    protos = _prototypes()
    assert len(protos) == len(_declared_functions())
    for name, (ret, params) in protos.items():
        assert name in l1._sig, name
        res, args = l1._sig[name]
        assert len(args) == len(params), (name, params)
        if ret == "void":
            assert res is None, name
        elif ret == "char *":
            assert res is ctypes.c_char_p, name
        else:
            assert ctypes.sizeof(res) == ctypes.sizeof(scalars[ret]), name
        for t, a in zip(params, args):
            if t.endswith("*"):
                assert a is ctypes.c_void_p or issubclass(a, ctypes._Pointer), (name, t)
            else:
                assert ctypes.sizeof(a) == ctypes.sizeof(scalars[t]), (name, t)
                assert issubclass(a, ctypes.c_double) == (t == "double"), (name, t)


def _unbound_instance(m, n):
    """An Instance object with sizes only: the checks below fire before any library call."""
    import paper_1503_03520_gb300 as l1
    inst = object.__new__(l1.Instance)
    inst._h = None
    inst.m, inst.n, inst.nnz = m, n, 0
    return inst


def test_binding_checks_vector_lengths_without_gpu():
    import numpy as np
    inst = _unbound_instance(10, 5)
    with pytest.raises(ValueError):
        inst.matvec(np.zeros(4))                      # A x needs n = 5 entries
    with pytest.raises(ValueError):
        inst.matvec(np.zeros(5), np.zeros(9))        # and writes m = 10
    with pytest.raises(ValueError):
        inst.rmatvec(np.zeros(5))                     # A^T y needs m = 10
    with pytest.raises(ValueError):
        inst.rmatvec(np.zeros(10), np.zeros(4))


def test_noalloc_binding_refuses_host_vectors_without_gpu():
    import numpy as np
    import torch
    inst = _unbound_instance(10, 5)
    with pytest.raises(ValueError, match="CUDA tensors"):
        inst.rmatvec_noalloc(np.zeros(10), np.zeros(5))
    with pytest.raises(ValueError, match="CUDA tensors"):
        inst.rmatvec_noalloc(torch.zeros(10), torch.zeros(5))
