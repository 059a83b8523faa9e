"""The C-ABI library builds, loads and exports every symbol of include/hsg.h;
argument checks that happen on the host before any CUDA call (CPU only)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hsg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:hsg_status|const char\*|int)\s+(hsg_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_1006_2566_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("hsg_create", "hsg_set_couplings", "hsg_sweep", "hsg_energy", "hsg_destroy"):
        assert n in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(lib):
    from paper_1006_2566_gb300 import build

    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (hsg_\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        getattr(lib, n)


def test_binding_wraps_every_declared_function(lib):
    from paper_1006_2566_gb300 import hsg

    for n in declared_functions():
        assert n in hsg._SIGS, n
        assert hasattr(hsg, n), n


def test_host_side_argument_checks(lib):
    from paper_1006_2566_gb300 import hsg

    assert hsg.hsg_version() == 100
    for L in (0, 2, 5, 7, 1625, 1626, -4):
        with pytest.raises(hsg.HsgError) as e:
            hsg.hsg_create(L, seed=1)
        assert e.value.status == hsg.HSG_EINVAL
        assert "L must be even" in hsg.hsg_last_error(None)
    assert hsg._lib.hsg_create(None, 8, 1, 0, 0, None) == hsg.HSG_EINVAL
    # the key's stream number 2*sample + replica must name each pair once:
    # (s, 2) would share every random number with (s + 1, 0), and sample
    # 2^31 + s with sample s
    for sample, replica in ((0, 2), (5, 3), (2 ** 31, 0), (2 ** 32 - 1, 1)):
        with pytest.raises(hsg.HsgError) as e:
            hsg.hsg_create(8, seed=1, sample=sample, replica=replica)
        assert e.value.status == hsg.HSG_EINVAL
        assert "replica must be 0 or 1" in hsg.hsg_last_error(None)
        out = ctypes.c_void_p(16)  # aligned, never written: the check comes first
        assert hsg._lib.hsg_philox(1, sample, replica, 0, 0, 0, 4, out, None) == hsg.HSG_EINVAL
    assert hsg._lib.hsg_test_fail_alloc(-1) == hsg.HSG_EINVAL
    assert hsg._lib.hsg_test_fail_alloc(0) == hsg.HSG_OK
    assert hsg._lib.hsg_test_stall_tensor_loads(4) == hsg.HSG_EINVAL
    assert hsg._lib.hsg_test_stall_tensor_loads(-1) == hsg.HSG_EINVAL
    assert hsg._lib.hsg_test_stall_tensor_loads(0) == hsg.HSG_OK
    # NULL / misaligned outputs are refused before any launch
    assert hsg._lib.hsg_philox(1, 0, 0, 0, 0, 0, 4, None, None) == hsg.HSG_EINVAL
    assert hsg._lib.hsg_philox(1, 0, 0, 0, 0, 0, 4, ctypes.c_void_p(8), None) == hsg.HSG_EINVAL
    # every entry point taking a context refuses NULL
    sch = hsg.schedule()
    assert hsg._lib.hsg_sweep(None, ctypes.byref(sch), 1) == hsg.HSG_EINVAL
    assert hsg._lib.hsg_energy(None, None) == hsg.HSG_EINVAL
    assert hsg._lib.hsg_set_couplings(None, None, 0, 0) == hsg.HSG_EINVAL
    assert hsg._lib.hsg_half_sweep(None, ctypes.byref(sch), 3, 0) == hsg.HSG_EINVAL
    assert hsg._lib.hsg_destroy(None) == hsg.HSG_OK
    assert hsg._lib.hsg_status_string(2) == b"HSG_ENOMEM"


def test_create_without_a_device_reports_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1006_2566_gb300 import hsg

    with pytest.raises(hsg.HsgError) as e:
        hsg.hsg_create(8, seed=1)
    assert e.value.status == hsg.HSG_ECUDA
