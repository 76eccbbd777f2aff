"""The C-ABI library loads and exports every function include/swepi.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "swepi.h")).read()
    return sorted(set(re.findall(r"\b(sw_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_boundary_calls():
    names = declared()
    for call in ("sw_init", "sw_rhs", "sw_jvp", "sw_kiops_phi", "sw_epi_step", "sw_free"):
        assert call in names


def test_library_exports_every_declared_symbol():
    from paper_2101_05617_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    lib = ctypes.CDLL(b.LIB)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2101_05617_gb300 import swepi
    assert sorted(swepi.EXPORTED) == sorted(n for n in declared())


def test_status_strings_without_gpu():
    from paper_2101_05617_gb300 import swepi
    assert swepi.sw_status_str(0) == "ok"
    assert "invalid" in swepi.sw_status_str(-1)


def test_argument_checks_without_gpu():
    """Host-side argument validation returns a status before any CUDA call:
    every call rejects a NULL context (or a bad size) with SW_EINVAL (-1), the
    queries return -1, and sw_free accepts NULL."""
    from paper_2101_05617_gb300 import swepi
    L = swepi.lib()
    EINVAL = -1
    prm = swepi.sw_params(6.37122e6, 9.80616, 7.292e-5, 0.0, 0.0, 0.0, 0)
    h = ctypes.c_void_p()
    assert L.sw_init(0, 3, ctypes.byref(prm), ctypes.byref(h)) == EINVAL and not h.value
    assert L.sw_init(4, 8, ctypes.byref(prm), ctypes.byref(h)) == EINVAL and not h.value   # p <= 7
    assert L.sw_init(4, 3, None, ctypes.byref(h)) == EINVAL
    for prec in (-1, 2):                                    # precision: 0 = FP64, 1 = complex64-bulk form
        bad = swepi.sw_params(6.37122e6, 9.80616, 7.292e-5, 0.0, 0.0, 0.0, prec)
        assert L.sw_init(4, 3, ctypes.byref(bad), ctypes.byref(h)) == EINVAL and not h.value
    x = ctypes.c_void_p(16)   # never dereferenced: every call below fails its NULL-context check first
    o = swepi.make_opts()
    st = swepi.sw_kiops_stats()
    assert L.sw_rhs(None, x, x, None) == EINVAL
    assert L.sw_jvp(None, x, x, 1e-30, x, None) == EINVAL
    assert L.sw_jvp_static_scratch(None, x, x, 1e-30, x, None) == EINVAL
    assert L.sw_linearize(None, x, None) == EINVAL
    assert L.sw_jvp_linearized(None, x, x, None) == EINVAL
    assert L.sw_kiops_phi(None, x, 1.0, 1.0, 1, None, ctypes.byref(o), x, ctypes.byref(st), None) == EINVAL
    assert L.sw_epi_step(None, 4, 900.0, x, ctypes.byref(o), ctypes.byref(st), None) == EINVAL
    assert L.sw_epi_step_host(None, 4, 900.0, x, ctypes.byref(o), ctypes.byref(st), None) == EINVAL
    assert L.sw_epi_set_history(None, 1, x, x, None) == EINVAL
    assert L.sw_epi_reset(None) == EINVAL
    nb = ctypes.c_size_t(0)
    assert L.sw_epi_checkpoint_size(None, ctypes.byref(nb)) == EINVAL
    assert L.sw_epi_checkpoint_save(None, x, 1 << 20, None) == EINVAL
    assert L.sw_epi_checkpoint_load(None, x, 1 << 20, None) == EINVAL
    assert L.sw_set_jvp_mode(None, 1) == EINVAL and L.sw_set_kiops_driver(None, 1) == EINVAL
    assert L.sw_set_orth_fused(None, 1, None) == EINVAL
    assert L.sw_set_bottom(None, x) == EINVAL and L.sw_set_bottom_host(None, x) == EINVAL
    assert L.sw_node_xyz(None, x) == EINVAL
    assert L.sw_state_from_fields(None, x, x, x, x) == EINVAL
    assert L.sw_diagnostics(None, x, x, None, None) == EINVAL
    assert L.sw_error_norms(None, x, x, x, None) == EINVAL
    assert L.sw_profile(None, 1) == EINVAL and L.sw_profile_kinds(None, 1) == EINVAL
    assert L.sw_profile_every(None, 4) == EINVAL
    assert L.sw_check_inject(None, 1) == EINVAL
    checked = ctypes.c_int(-1)
    assert L.sw_check_status(ctypes.byref(checked)) == 0 and checked.value == 0   # default build: no checks
    assert L.sw_fp64_fma_peak(None) == EINVAL
    assert L.sw_set_controller(None, None) == EINVAL
    assert L.sw_kiops_log(None, None, 0) == EINVAL
    assert L.sw_mlp_forward(None, x, 1, x, None) == EINVAL
    assert L.sw_ens_create(0, None, ctypes.byref(h)) == EINVAL
    assert L.sw_ens_free(None) == EINVAL and L.sw_ens_set_policy(None, 0.5) == EINVAL
    assert L.sw_num_unknowns(None) == -1 and L.sw_kernel_launches(None) == -1
    L.sw_free(None)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2101_05617_gb300 import swepi
    monkeypatch.setattr(swepi, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(swepi, "_lib", None)
    with pytest.raises(ImportError):
        swepi.lib()
