"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/gmm_gb300.h declares.  No GPU needed."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names.update(re.findall(r"\b(gmm_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1707_09094_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    declared = _declared()
    assert {"gmm_learn", "gmm_log_p", "gmm_assign", "gmm_em_iterate"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gmm_[a-z0-9_]+)", out))
    assert declared <= exported, declared - exported
    lib = ctypes.CDLL(libpath)
    for n in declared:
        getattr(lib, n)


def test_binding_names_match_header():
    from paper_1707_09094_gb300 import _lib
    assert set(_lib.SIGNATURES) <= _declared()


def test_default_opts_and_error_text(libpath):
    from paper_1707_09094_gb300 import _lib
    lib = _lib.load()
    o = _lib.gmm_learn_opts()
    lib.gmm_default_opts(ctypes.byref(o))
    assert (o.dist, o.seed_mode, o.seed, o.em_tol, o.prec, o.print) == (_lib.GMM_MAHA, _lib.GMM_RANDOM_SUBSET,
                                                                        0, 0.0, _lib.GMM_FP32, 0)
    assert isinstance(lib.gmm_last_error(), bytes)


def test_null_model_arguments_are_rejected_without_touching_the_gpu(libpath):
    from paper_1707_09094_gb300 import _lib
    lib = _lib.load()
    assert lib.gmm_learn(None, None, 10, 2, 2, 1, 1, 1e-10, None) == _lib.GMM_ERR_ARG
    assert lib.gmm_em_iterate(None, None, 10, 1, 1e-10, 0, 0, None) == _lib.GMM_ERR_ARG
    assert lib.gmm_get_stats(None, None, 0, None) == _lib.GMM_ERR_ARG
    assert lib.gmm_create(None) == _lib.GMM_ERR_ARG
    lib.gmm_destroy(None)


def test_kernels_are_built_for_sm103a_only(libpath):
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    archs = set(re.findall(r"sm_(\d+a?)", out.stdout))
    assert archs == {"103a"}, archs


def test_binding_constants_match_header():
    """Every GMM_* integer the binding defines has the header's value."""
    from paper_1707_09094_gb300 import _lib
    src = ""
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src += open(os.path.join(inc, f)).read()
    header = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(GMM_[A-Z0-9_]+)\s+(-?\d+)\b", src)}
    header.update({m.group(1): int(m.group(2)) for m in re.finditer(r"\b(GMM_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)})
    mine = {k: v for k, v in vars(_lib).items() if k.startswith("GMM_") and isinstance(v, int)}
    assert mine, "the binding defines no GMM_* constants"
    for k, v in mine.items():
        if k in header:
            assert header[k] == v, (k, header[k], v)
    assert {"GMM_DEBUG_TC_FORM", "GMM_DEBUG_FP32_FORM", "GMM_STAT_SCREENED"} <= set(mine) & set(header)
