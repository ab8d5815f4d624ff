"""The C ABI boundary, checked without a GPU: every function include/ising.h
declares is exported by libising.so and has a ctypes signature in the
binding, and the host-only entry points behave."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ising_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1811_04384_gb300 import build
    build.build()
    import paper_1811_04384_gb300 as p
    return p.load()


def test_header_matches_binding():
    from paper_1811_04384_gb300 import SYMBOLS
    assert header_functions() == set(SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    from paper_1811_04384_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = header_functions() - exported
    assert not missing, missing
    for name in header_functions():
        assert hasattr(lib, name)


def test_host_only_entry_points(lib):
    import paper_1811_04384_gb300 as p
    assert lib.ising_strerror(0) == b"ok"
    assert lib.ising_strerror(p.ISING_EINVAL) == b"invalid argument"
    assert lib.ising_strerror(12345) == b"unknown error code"
    for bad in (0, 2, 3, 5, 33, 32770, -4):
        assert lib.ising_bytes_required(bad) == 0
    # two colour arrays of L x pitch words (pitch = W rounded up to even)
    for L, W in ((4, 1), (42, 1), (44, 2), (64, 2), (1024, 25), (16384, 391), (32768, 781)):
        P = W + (W & 1)
        assert lib.ising_bytes_required(L) >= 2 * L * P * 8
        assert lib.ising_bytes_required(L) < 2 * L * P * 8 + (1 << 20)
    assert lib.ising_destroy(None) == 0
    # the normal build checks no indices: the status call touches no device
    assert p.check_status() == (False, 0)


def test_invalid_arguments_are_rejected_before_any_device_call(lib):
    import ctypes
    import paper_1811_04384_gb300 as p
    h = ctypes.c_void_p()
    assert lib.ising_create(7, 1, ctypes.byref(h)) == p.ISING_EINVAL
    assert lib.ising_create(2, 1, ctypes.byref(h)) == p.ISING_EINVAL
    assert lib.ising_create(65536, 1, ctypes.byref(h)) == p.ISING_EINVAL
    assert lib.ising_create(64, 1, None) == p.ISING_EINVAL
    assert lib.ising_sweep(None, 1) == p.ISING_EINVAL
    assert lib.ising_set_beta(None, 0.5) == p.ISING_EINVAL
    assert lib.ising_set_path(None, p.ISING_PATH_CLUSTER) == p.ISING_EINVAL
    assert lib.ising_set_clusters(None, 2) == p.ISING_EINVAL
    assert lib.ising_cluster_inject_stall(None, 1) == p.ISING_EINVAL
    assert lib.ising_cluster_inject_absent(None, 0) == p.ISING_EINVAL
    path = ctypes.c_int32(-1)
    assert lib.ising_get_path(None, ctypes.byref(path)) == p.ISING_EINVAL and path.value == -1
    assert lib.ising_philox_blocks(1, None, None, 4) == p.ISING_EINVAL
    # the serving entry points of the boundary, in the two-argument form
    assert lib.ising_server_create(1 << 20, None) == p.ISING_EINVAL
    assert lib.ising_server_create(255, ctypes.byref(h)) == p.ISING_EINVAL
    assert lib.ising_server_create_ex(1 << 20, 0, 50, ctypes.byref(h)) == p.ISING_EINVAL
    assert lib.ising_server_create_ex(1 << 20, 256, 1 << 17, ctypes.byref(h)) == p.ISING_EINVAL
    assert lib.ising_server_inject_fault(None, 0) == p.ISING_EINVAL
    assert lib.ising_strerror(p.ISING_EINTERNAL) == b"internal host error in the server worker"


def test_product_path_has_no_oracle_dependency():
    """The package never imports, links or runs anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_1811_04384_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "oracle.c" not in text and "liboracle" not in text, fn


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libising.so the binding raises instead of falling back."""
    import paper_1811_04384_gb300 as p
    monkeypatch.setattr(p, "_lib", None)
    monkeypatch.setattr(p, "LIB_PATH", str(tmp_path / "libising.so"))
    with pytest.raises(ImportError, match="no CPU fallback"):
        p.load()
    with pytest.raises(ImportError):
        p.Lattice(64, 1)
