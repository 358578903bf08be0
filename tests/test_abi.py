"""The C-ABI library builds, loads and exports every entry point declared in
include/sdsl.h (no GPU needed: nothing here launches a kernel)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "sdsl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sdsl_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_23979_gb300 import build, sdsl

    build.build()
    return sdsl.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("sdsl_setup", "sdsl_factor", "sdsl_solve", "sdsl_update_diag", "sdsl_free"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, f"not exported: {missing}"


def test_host_only_entry_points(lib):
    """Calls that need no device: defaults, status strings, NULL handling."""
    from paper_2604_23979_gb300 import sdsl

    o = sdsl.sdsl_default_options()
    assert o.tau == 1e-3 and o.delta == 1e-12 and o.rtol == 1e-8 and o.maxit == 2000 and o.restart == 30
    assert o.factor_prec == 64 and o.refactor_ratio == 1.5
    assert lib.sdsl_status_str(0) == b"ok"
    assert lib.sdsl_status_str(5) == b"not converged"
    assert lib.sdsl_free(None) == 0
    assert lib.sdsl_factor(None) == sdsl.ERR_ARG
    assert lib.sdsl_solve(None, None, None, 1, None) == sdsl.ERR_ARG
    import ctypes
    h = ctypes.c_void_p()
    assert lib.sdsl_setup(None, 1, 1, None, None, None, None, ctypes.byref(h)) == sdsl.ERR_ARG
    assert h.value is None
    # option validation happens before any device work
    o.factor_prec = 8
    assert lib.sdsl_setup(ctypes.byref(o), 1, 1, None, None, None, None, ctypes.byref(h)) == sdsl.ERR_ARG
    assert b"factor_prec" in lib.sdsl_last_error()


def test_struct_layouts_match_header(lib):
    """ctypes mirrors of the ABI structs have the field order of the header."""
    from paper_2604_23979_gb300 import sdsl

    text = open(os.path.join(ROOT, "include", "sdsl.h")).read()
    for struct, cls in (("sdsl_options", sdsl.sdsl_options), ("sdsl_stats", sdsl.sdsl_stats),
                        ("sdsl_info", sdsl.sdsl_info)):
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + struct + ";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            for part in decl.split(","):
                part = re.sub(r"\[[^\]]*\]", "", part.strip())  # arrays: keep the name
                names.append(re.findall(r"([A-Za-z_][A-Za-z_0-9]*)\s*$", part.strip())[0])
        assert names == [f for f, _ in cls._fields_], struct


def test_enum_values_match_header():
    """The binding's status, form, method and memory-space constants equal the
    header's enumerators."""
    from paper_2604_23979_gb300 import sdsl

    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "sdsl.h")).read(), flags=re.S)
    values = {}
    for body in re.findall(r"enum\s*\{([^}]*)\}", text):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            name, _, val = item.partition("=")
            nxt = int(val) if val.strip() else nxt
            values[name.strip()] = nxt
            nxt += 1
    pairs = {"SDSL_OK": sdsl.OK, "SDSL_ERR_ARG": sdsl.ERR_ARG, "SDSL_ERR_OOM": sdsl.ERR_OOM,
             "SDSL_ERR_CUDA": sdsl.ERR_CUDA, "SDSL_ERR_BREAKDOWN": sdsl.ERR_BREAKDOWN,
             "SDSL_ERR_NOT_CONVERGED": sdsl.ERR_NOT_CONVERGED, "SDSL_ERR_TIMEOUT": sdsl.ERR_TIMEOUT,
             "SDSL_ERR_STATE": sdsl.ERR_STATE, "SDSL_FORM_CSR": sdsl.FORM_CSR, "SDSL_FORM_NORMAL": sdsl.FORM_NORMAL,
             "SDSL_FORM_AUGMENTED": sdsl.FORM_AUGMENTED, "SDSL_BJ_PCG": sdsl.BJ_PCG,
             "SDSL_BBD_GMRES": sdsl.BBD_GMRES, "SDSL_BJ_BICGSTAB": sdsl.BJ_BICGSTAB, "SDSL_BBD_GCR": sdsl.BBD_GCR,
             "SDSL_MEM_HOST": sdsl.MEM_HOST, "SDSL_MEM_DEVICE": sdsl.MEM_DEVICE}
    for name, v in pairs.items():
        assert values.get(name) == v, (name, values.get(name), v)
