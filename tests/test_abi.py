"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/mpjsvd.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "mpjsvd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mpjsvd_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2209_04626_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["mpjsvd_create", "mpjsvd_svd", "mpjsvd_svd_batched", "mpjsvd_svd_backward",
                     "mpjsvd_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_2209_04626_gb300 import mpjsvd
    assert sorted(mpjsvd.EXPORTS) == _declared()
    for name in _declared():
        assert callable(getattr(mpjsvd, name))


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of mpjsvd_params / mpjsvd_stats have the C layout: gcc compiles the
    header and reports sizeof and offsetof of every field."""
    import subprocess
    from paper_2209_04626_gb300 import mpjsvd
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mpjsvd.h"', "int main(void) {"]
    for cname, cls in (("mpjsvd_params", mpjsvd.Params), ("mpjsvd_stats", mpjsvd.Stats)):
        lines.append('printf("%%s %%zu\\n", "%s", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%%s.%%s %%zu\\n", "%s", "%s", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.split("\n") if l)
    for cname, cls in (("mpjsvd_params", mpjsvd.Params), ("mpjsvd_stats", mpjsvd.Stats)):
        assert int(out[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(out["%s.%s" % (cname, f)]) == getattr(cls, f).offset, (cname, f)


def test_default_params_are_the_papers(lib_path):
    """The tunables of Section 7.1 and the documented defaults of the algorithm choices
    (host only: mpjsvd_default_params makes no CUDA call)."""
    from paper_2209_04626_gb300 import mpjsvd
    p = mpjsvd.mpjsvd_default_params()
    assert (p.tol_alg, p.tol_orth, p.tol_cond_coef) == (1e-2, 1e-5, 1.5)
    assert p.trailing_frac == 0.25 and p.maxsweep == 30 and p.block_w == 0
    assert p.mode == 0 and p.precond == 0 and p.qr_first == 0 and p.qrcp == 0 and p.stop == 0
    # the kernel choices default to the automatic ones (by size), the options of Section 3.4 off
    assert p.wait_limit_ms == 4000 and p.low_kernel == 0 and p.gemm_kernel == 0
    assert p.work_kernel == 0 and p.work_cluster == 0 and p.qr_update == 0
    assert p.v_by_qr == 0 and p.switch_method == 0 and p.y_tol == 0.0


def test_argument_validation_without_gpu(lib_path):
    """Invalid arguments are rejected before any CUDA call (LAPACK-style -i codes)."""
    lib = ctypes.CDLL(lib_path)
    f = lib.mpjsvd_svd
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]
    assert f(None, 4, 2, None, 4, None, None, None, 0.0) == -1
    lib.mpjsvd_default_params.argtypes = [ctypes.c_void_p]
    assert lib.mpjsvd_default_params(None) == -1


def test_python_choice_names_match_the_header_constants(lib_path):
    """Every name the binding accepts for an algorithm choice maps to the value of the header's
    #define of the same choice (MPJSVD_<GROUP>_<NAME>), and every such #define has a name."""
    import re
    from paper_2209_04626_gb300 import mpjsvd
    hdr = open(os.path.join(ROOT, "include", "mpjsvd.h")).read()
    groups = {"MODE": mpjsvd.MODE, "PRECOND": mpjsvd.PRECOND, "QRCP": mpjsvd.QRCP, "STOP": mpjsvd.STOP,
              "LOWK": mpjsvd.LOWK, "SWITCH": mpjsvd.SWITCH, "GEMMK": mpjsvd.GEMMK, "WORKK": mpjsvd.WORKK,
              "QRU": mpjsvd.QRU}
    aliases = {"RT": "rt", "ALG1": "alg1", "XGESVJ": "xgesvj", "REG": "reg", "CTA": "cta"}
    for g, names in groups.items():
        defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define MPJSVD_%s_(\w+) (\d+)" % g, hdr)}
        assert defs, g
        assert sorted(defs.values()) == sorted(names.values()), (g, defs, names)
        for cname, val in defs.items():
            key = aliases.get(cname, cname.lower())
            assert names.get(key) == val, (g, cname, key, names)
        # and the binding maps them into the params struct
        field = {"MODE": "mode", "PRECOND": "precond", "QRCP": "qrcp", "STOP": "stop", "LOWK": "low_kernel",
                 "SWITCH": "switch_method", "GEMMK": "gemm_kernel", "WORKK": "work_kernel", "QRU": "qr_update"}[g]
        for key, val in names.items():
            assert getattr(mpjsvd.mpjsvd_default_params(**{field: key}), field) == val
