"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads, and
exports every entry point that include/hzb.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "hzb.h")).read()
    return re.findall(r"^\s*(?:hzb_status|void|const char \*)\s*\*?(hzb_\w+)\(", txt, re.M)


def test_header_declares_the_boundary():
    names = set(declared_symbols())
    for n in ("hzb_create", "hzb_destroy", "hzb_set_wave", "hzb_add_body", "hzb_build_scattering_matrices",
              "hzb_solve_plane_waves", "hzb_solve_data", "hzb_get_density", "hzb_far_field", "hzb_apply",
              "hzb_interbody", "hzb_local_inverse", "hzb_eval_field", "hzb_last_error",
              "hzb_save_scattering", "hzb_load_scattering", "hzb_add_body_curve",
              "hzb_compress", "hzb_set_skeleton", "hzb_get_skeleton", "hzb_set_acceleration",
              "hzb_reduced_size", "hzb_apply_reduced", "hzb_interp_decomp", "hzb_measure_peak",
              "hzb_local_inverse_noalloc"):
        assert n in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_1406_0236_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1406_0236_gb300.binding as bd
    monkeypatch.setattr(bd, "_LIBPATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(bd, "_lib", None)
    try:
        bd.lib()
    except ImportError:
        return
    raise AssertionError("missing library did not raise")


def test_status_strings_and_default_options_without_gpu():
    from paper_1406_0236_gb300 import binding as bd
    L = bd.lib()
    o = bd._Options()
    L.hzb_default_options(ctypes.byref(o))
    assert o.precision == 0 and abs(o.gmres_tol - 1e-10) < 1e-25 and o.maxit == 500
    assert L.hzb_status_string(-4) == b"GMRES did not converge"
