"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/amg.h declares (no compute calls here)."""
import ctypes
import os
import re
import shutil

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "amg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(amg_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1512_04629_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["amg_setup", "amg_sparsify", "amg_reintroduce", "amg_solve", "amg_solve_batch",
                     "amg_level_stats", "amg_hierarchy_save", "amg_hierarchy_load", "amg_free",
                     "amg_status_str", "amg_last_error", "amg_server_create", "amg_server_register",
                     "amg_server_submit", "amg_server_wait", "amg_server_destroy"]:
        assert required in names, required


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.amg_status_str.restype = ctypes.c_char_p
    assert lib.amg_status_str(0) == b"AMG_OK"
    assert lib.amg_status_str(8) == b"AMG_REJECTED"


def test_binding_signatures_cover_header():
    from paper_1512_04629_gb300 import amg

    assert set(declared_functions()) == set(amg.SIGNATURES)


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    from paper_1512_04629_gb300 import amg

    monkeypatch.setattr(amg, "_lib", None)
    monkeypatch.setattr(amg, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        amg.lib()


def header_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/amg.h, in order."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text, flags=re.S)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        parts = [p.strip() for p in decl.split(",") if p.strip()]
        for p in parts:  # "int32_t nrows" / "ncols" / "const int32_t *rowptr"
            fields.append(re.findall(r"[A-Za-z_][A-Za-z0-9_]*", p)[-1])
    return fields


@pytest.mark.parametrize("cname,pyname", [("amg_options", "Options"), ("amg_solve_info", "SolveInfo"),
                                          ("amg_level_info", "LevelInfo"), ("amg_server_opts", "ServerOpts")])
def test_binding_structs_mirror_header(cname, pyname):
    from paper_1512_04629_gb300 import amg

    assert [f for f, _ in getattr(amg, pyname)._fields_] == header_struct_fields(cname)


def test_option_defaults_without_gpu(libpath):
    from paper_1512_04629_gb300 import amg

    o = amg.default_options()
    assert (o.theta, o.max_size, o.max_levels, o.method, o.precision) == (0.25, 100, 25, amg.METHOD_SPARSE, 0)
    assert (o.lump, o.krylov, o.restart) == (amg.LUMP_DIAG, amg.KRYLOV_CG, 30)
    assert (o.k_check, o.s_levels, o.gamma_min, o.rho_max) == (3, 1, 0.01, 0.5)
    assert o.div_factor == 1e3 and o.transfer_variant == amg.SPMV_AUTO
    so = amg.ServerOpts()
    amg.lib().amg_server_opts_default(ctypes.byref(so))
    assert (so.max_batch, so.hbm_budget, so.max_queue, so.max_it, so.stage_budget) == (32, 0, 4096, 500, 0)
    assert so.wait_limit_ms == 120000


@pytest.mark.parametrize("field,value", [("max_batch", 0), ("max_batch", 65), ("max_queue", 0), ("max_it", 0),
                                         ("hbm_budget", -1), ("stage_budget", -2), ("wait_limit_ms", 0)])
def test_server_options_rejected_before_any_cuda_call(libpath, field, value):
    from paper_1512_04629_gb300 import amg

    L = amg.lib()
    o = amg.ServerOpts()
    L.amg_server_opts_default(ctypes.byref(o))
    setattr(o, field, value)
    out = ctypes.c_void_p()
    assert L.amg_server_create(ctypes.byref(o), ctypes.byref(out)) == amg.ERR_INVALID
    assert not out.value
    assert b"out of range" in L.amg_last_error()


@pytest.mark.parametrize("theta,kw,gamma,msg", [
    (1.5, {}, None, "theta"), (float("nan"), {}, None, "theta"),
    (0.25, dict(max_size=0), None, "max_size"), (0.25, dict(max_levels=0), None, "max_levels"),
    (0.25, dict(max_levels=65), None, "max_levels"), (0.25, dict(method=9), None, "method"),
    (0.25, dict(precision=7), None, "precision"), (0.25, dict(k_check=0), None, "k_check"),
    (0.25, dict(check_every=0), None, "check_every"), (0.25, dict(lump=4), None, "lump"),
    (0.25, dict(krylov=3), None, "krylov"), (0.25, dict(restart=0), None, "restart"),
    (0.25, dict(restart=513), None, "restart"), (0.25, dict(div_factor=0.5), None, "div_factor"),
    (0.25, dict(div_factor=float("inf")), None, "div_factor"), (0.25, dict(spmv_variant=10), None, "spmv_variant"),
    (0.25, dict(transfer_variant=10), None, "transfer_variant"),
    (0.25, {}, [0.5, 0.1], "level 0 is never sparsified"), (0.25, {}, [0.0, float("nan")], "finite"),
    (0.25, {}, [0.0, -0.1], ">= 0"),
])
def test_setup_rejects_bad_arguments_before_any_cuda_call(libpath, theta, kw, gamma, msg):
    import amg_inputs as gen
    from paper_1512_04629_gb300 import amg

    A = gen.poisson2d_5pt(6)
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy.setup(A, theta=theta, gamma=gamma, **kw)
    assert e.value.status == amg.ERR_INVALID
    assert msg in str(e.value)


def test_setup_rejects_a_non_square_matrix(libpath):
    import numpy as np

    from paper_1512_04629_gb300 import amg

    rp = np.array([0, 1, 2], dtype=np.int32)
    A = amg.csr_struct(rp, np.array([0, 2], dtype=np.int32), np.array([1.0, 1.0]), ncols=3)
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy.setup(A)
    assert e.value.status == amg.ERR_INVALID and "square" in str(e.value)
