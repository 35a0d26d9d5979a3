"""The C-ABI library loads and exports every entry point include/gmcs.h
declares, the binding declares the same set, and the struct layouts agree.
No GPU work is done here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gmcs.h")
DIAG_HEADER = os.path.join(ROOT, "include", "gmcs_diag.h")


def declared(header=HEADER):
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gmcs_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ["gmcs_create", "gmcs_destroy", "gmcs_init_particles", "gmcs_add_keyframe", "gmcs_step",
              "gmcs_eval", "gmcs_move", "gmcs_predict", "gmcs_select", "gmcs_weigh", "gmcs_resample",
              "gmcs_get_particles", "gmcs_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2504_18056_b300 import build
    build.build()
    lib = C.CDLL(build.OUT)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_2504_18056_b300 as g
    assert sorted(g._SIGS) == declared()


def test_diagnostics_live_in_their_own_library():
    """Calibration probes are not part of the particle-update ABI: libgmcs.so does
    not export them, libgmcs_diag.so exports what gmcs_diag.h declares."""
    import paper_2504_18056_b300 as g
    from paper_2504_18056_b300 import build
    build.build()
    names = declared(DIAG_HEADER)
    assert names == sorted(g._DIAG_SIGS) == ["gmcs_probe_ffma", "gmcs_probe_gather"]
    assert not set(names) & set(declared())
    main, diag = C.CDLL(build.OUT), C.CDLL(build.DIAG_OUT)
    assert all(hasattr(diag, n) for n in names)
    assert not any(hasattr(main, n) for n in names)


def test_struct_sizes_and_defaults():
    import paper_2504_18056_b300 as g
    assert C.sizeof(g.Config) == 104
    assert C.sizeof(g.StepOut) == 152
    assert C.sizeof(g.Grid) == 48
    cfg = g.default_config()
    assert cfg.k_nb == 3 and cfg.steps == 3 and abs(cfg.sigma - 0.2) < 1e-7 and abs(cfg.r_t - 1.0) < 1e-7
    assert abs(cfg.prune_w - 1e-8) < 1e-15 and abs(cfg.prune_lr - 1e-16) < 1e-23
    assert cfg.kf_overlap == 0.0 and cfg.kf_voxel == 1.0 and abs(cfg.kf_h - 0.2) < 1e-7
    assert cfg.model == g.MODEL_FIELD and cfg.knn == 10 and abs(cfg.cov_eps - 1e-3) < 1e-9 and cfg.gicp_tau == 20.0
    assert g.strerror(g.E_CAPACITY) == "capacity exceeded"


def test_invalid_arguments_are_rejected_without_a_device():
    import paper_2504_18056_b300 as g
    out = C.c_void_p()
    cfg = g.default_config(k_nb=0)
    assert g.lib().gmcs_create(C.byref(cfg), 10, 1, 10, None, C.byref(out)) == g.E_INVALID
    cfg = g.default_config()
    assert g.lib().gmcs_create(C.byref(cfg), 0, 1, 10, None, C.byref(out)) == g.E_INVALID
    assert g.lib().gmcs_create(None, 10, 1, 10, None, C.byref(out)) == g.E_INVALID
    assert g.lib().gmcs_destroy(None) == g.OK
