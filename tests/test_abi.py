"""The C-ABI library builds, loads and exports every entry point include/recon.h declares, and
the Python binding marshals the same names (no GPU needed: nothing here launches work)."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "recon.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(recon_[a-z_0-9]+)\s*\(", src)))


def _cuda_visible():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return os.path.exists("/dev/nvidiactl")


@pytest.fixture(scope="module")
def lib():
    from paper_1704_04511_gb300 import build, recon
    build.build()
    return recon.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "recon_solve" in names and "recon_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header(lib):
    from paper_1704_04511_gb300 import recon
    assert sorted(recon.EXPORTED) == _declared()
    for n in recon.EXPORTED:
        assert callable(getattr(recon, n))


def test_bytes_needed_formula(lib):
    from paper_1704_04511_gb300 import recon
    small = recon.recon_bytes_needed((8, 32, 32), (5, 5, 2))
    big = recon.recon_bytes_needed((16, 256, 256), (9, 9, 3))
    assert 0 < small < big
    # three complex64 work vectors dominate at 256x256x16
    assert big >= 3 * 16 * 256 * 256 * 8
    assert recon.recon_bytes_needed((0, 32, 32), (5, 5, 2)) == 0


def test_profile_names(lib):
    from paper_1704_04511_gb300 import recon
    names = [recon.recon_profile_name(k) for k in range(recon.PROF_KINDS)]
    assert names[2] == "eig" and names[10] == "cg_update" and names[12] == "hpd_inverse"
    assert all(names)
    assert recon.recon_profile_name(recon.PROF_KINDS) == ""


def test_null_context_is_rejected(lib):
    from paper_1704_04511_gb300 import recon
    assert lib.recon_solve(None, recon.recon_dims(32, 32, 8), None, None,
                           recon.recon_filter(5, 5, 2), None, None) == recon.RECON_EINVAL


def test_binding_constants_match_header(lib):
    """Every integer #define the binding mirrors has the header's value."""
    from paper_1704_04511_gb300 import recon
    src = open(os.path.join(ROOT, "include", "recon.h")).read()
    defines = {m.group(1): int(m.group(2)) for m in
               re.finditer(r"#define (RECON_[A-Z0-9_]+) \(?(-?\d+)\)?", src)}
    mirrored = [n for n in dir(recon) if n.startswith("RECON_") and isinstance(getattr(recon, n), int)]
    assert "RECON_OPT_INJECT_BARRIER_FAULT" in mirrored and "RECON_ETIMEOUT" in mirrored
    for n in mirrored:
        if n in defines:
            assert getattr(recon, n) == defines[n], n
    assert recon.PROF_KINDS == defines["RECON_PROF_KINDS"]


def test_static_gram_checks_pointers_first(lib):
    """recon_gram_static refuses null or misaligned device pointers with RECON_EINVAL before it
    touches the device (the values are never dereferenced). The made-up addresses must never
    reach a GPU, so the test runs only in processes that see no CUDA device."""
    import ctypes
    if _cuda_visible():
        pytest.skip("a CUDA device is visible: made-up device addresses stay on device-less hosts")
    from paper_1704_04511_gb300 import recon
    d, f = recon.recon_dims(32, 32, 8), recon.recon_filter(5, 5, 2)
    assert lib.recon_gram_static(d, f, None, ctypes.c_void_p(4096), None, None) == recon.RECON_EINVAL
    assert lib.recon_gram_static(d, f, ctypes.c_void_p(4096 + 8), ctypes.c_void_p(8192), None,
                                 None) == recon.RECON_EINVAL
    assert lib.recon_gram_static(d, f, ctypes.c_void_p(4096), ctypes.c_void_p(8192),
                                 ctypes.c_void_p(16384 + 4), None) == recon.RECON_EINVAL
