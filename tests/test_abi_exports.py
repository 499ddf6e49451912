"""CPU checks of the boundary: the library builds for sm_103a, loads, exports
every symbol include/smf.h declares, and shares no code with the oracle."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "smf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(smf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libsmf():
    from paper_2605_19254_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = _declared()
    for n in ["smf_rns_reduce", "smf_residue_gemm", "smf_crt_reconstruct", "smf_rns_matmul",
              "smf_basis_create", "smf_create", "smf_destroy"]:
        assert n in names


def test_every_declared_symbol_is_exported(libsmf):
    from paper_2605_19254_gb300 import smf
    for name in _declared():
        assert hasattr(libsmf, name), name
    assert set(_declared()) == set(smf.EXPORTS)


def test_version_string(libsmf):
    libsmf.smf_version.restype = ctypes.c_char_p
    assert b"sm_103a" in libsmf.smf_version()


def test_no_device_calls_without_gpu_fail_cleanly(libsmf):
    # without a GPU, smf_create must refuse (no CPU fallback exists)
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    libsmf.smf_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_size_t]
    assert libsmf.smf_create(ctypes.byref(h), 0, 1, 0) != 0
    assert not h.value


def test_context_settings_reject_a_missing_context(libsmf):
    # host-only argument checks of the context settings: no context, or a
    # negative panel threshold, is SMF_E_INVALID, with nothing touched
    from paper_2605_19254_gb300 import smf
    P = ctypes.c_void_p
    libsmf.smf_set_elim_panels.argtypes = [P, ctypes.c_int64]
    libsmf.smf_set_fused_crt.argtypes = [P, ctypes.c_int]
    libsmf.smf_debug_inject.argtypes = [P, ctypes.c_int]
    libsmf.smf_profile_enable.argtypes = [P, ctypes.c_int]
    assert libsmf.smf_set_elim_panels(None, 0) == smf.SMF_E_INVALID
    assert libsmf.smf_set_elim_panels(None, -1) == smf.SMF_E_INVALID
    assert libsmf.smf_set_fused_crt(None, 1) == smf.SMF_E_INVALID
    assert libsmf.smf_debug_inject(None, 0) == smf.SMF_E_INVALID
    assert libsmf.smf_profile_enable(None, 1) == smf.SMF_E_INVALID


def test_oracle_and_cuda_path_share_nothing():
    csrc = glob.glob(os.path.join(ROOT, "paper_2605_19254_gb300", "**", "*"), recursive=True)
    for f in csrc:
        if os.path.isfile(f) and f.endswith((".cu", ".h", ".cpp", ".py")):
            text = open(f, errors="ignore").read()
            assert "oracle" not in re.sub(r"#.*|//.*", "", text).lower() or f.endswith("inputs.py"), f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".c", ".py")):
            text = open(f).read()
            assert "paper_2605_19254_gb300" not in text and "smf.h" not in text, f


def test_product_path_has_no_cpu_fallback(tmp_path, monkeypatch):
    from paper_2605_19254_gb300 import smf
    monkeypatch.setattr(smf, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(smf, "_lib", None)
    with pytest.raises(RuntimeError):
        smf.lib()
