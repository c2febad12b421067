"""The C-ABI library builds, loads and exports every entry point include/smppi.h
declares; host-side argument checks reject bad input before any device work
(these run without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "smppi.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2302_11719_gb300 import build as B
    path = B.build()
    return C.CDLL(path)


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(smppi_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared()
    for must in ("smppi_create", "smppi_destroy", "smppi_step", "smppi_update", "smppi_repair",
                 "smppi_cost_grad", "smppi_apply", "smppi_shield_update", "smppi_last_error",
                 "smppi_sync_status"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2302_11719_gb300 import smppi
    assert set(declared()) <= set(smppi._SIGS), set(declared()) - set(smppi._SIGS)


def test_default_params_and_host_checks(lib):
    from paper_2302_11719_gb300 import smppi
    smppi.load_library(os.path.join(ROOT, "paper_2302_11719_gb300", "libsmppi.so"))
    p = smppi.default_params()
    assert p.K == 256 and p.T == 50 and p.N_r == 50
    assert abs(p.m - 21.7) < 1e-5 and abs(p.lam - 1.0) < 1e-7 and abs(p.alpha - 0.3) < 1e-7
    assert abs(p.sigma[0] - 0.15) < 1e-7 and abs(p.sigma[1] - 0.3) < 1e-7
    L = smppi.load_library()
    h = C.c_void_p()
    # no track -> argument error, found on the host before any CUDA call
    assert L.smppi_create(C.byref(p), None, C.byref(h)) == smppi.ERR_ARG
    assert h.value is None
    assert b"track" in L.smppi_last_error(None)
    p.track_xy = 1234          # never dereferenced: the K check fails first
    p.n_track = 1024
    for field, bad in (("K", 0), ("T", 0), ("T", 513), ("N_r", 51), ("n_track", 2),
                       ("n_track", 4096), ("max_seq", 0)):
        q = smppi.default_params()
        C.memmove(C.byref(q), C.byref(p), C.sizeof(p))
        setattr(q, field, bad)
        assert L.smppi_create(C.byref(q), None, C.byref(h)) == smppi.ERR_ARG, field
    q = smppi.default_params()
    C.memmove(C.byref(q), C.byref(p), C.sizeof(p))
    q.lam = 0.0
    assert L.smppi_create(C.byref(q), None, C.byref(h)) == smppi.ERR_ARG
    assert b"lambda" in L.smppi_last_error(None)
    # the state kind: 0 or 1, and the curvilinear state needs C = 1.5 and |steer| <= 1/2
    assert p.state_kind == 0
    for kind, Ct, steer in ((2, 1.5, 0.5), (1, 1.2, 0.5), (1, 1.5, 0.6)):
        q = smppi.default_params()
        C.memmove(C.byref(q), C.byref(p), C.sizeof(p))
        q.state_kind, q.Ct, q.u_max[0] = kind, Ct, steer
        assert L.smppi_create(C.byref(q), None, C.byref(h)) == smppi.ERR_ARG
        assert b"state_kind" in L.smppi_last_error(None)
    # calls on a NULL handle are rejected
    assert L.smppi_step(None, None, None, 0, 0, None, None) == smppi.ERR_ARG
    assert L.smppi_repair(None, 1, None, None, None, 1, 1, C.c_float(0), None, None) == smppi.ERR_ARG
    assert L.smppi_destroy(None) == smppi.OK


def test_curvilinear_state_refused_where_unsupported(lib):
    """The batch and smppi_step_noalloc take the Cartesian state only: a valid
    state_kind 1 parameter set is refused on the host, before any device work."""
    from paper_2302_11719_gb300 import smppi
    smppi.load_library(os.path.join(ROOT, "paper_2302_11719_gb300", "libsmppi.so"))
    L = smppi.load_library()
    p = smppi.default_params()
    p.track_xy = 1234          # never dereferenced: the state kind is refused first
    p.n_track = 64
    p.state_kind = 1
    assert L.smppi_step_noalloc(C.byref(p), None, None, 0, 0, None, None) == smppi.ERR_ARG
    assert b"state_kind" in L.smppi_last_error(None)
    descs = (smppi.InstanceDesc * 1)()
    b = C.c_void_p()
    assert L.smppi_batch_create(C.byref(p), 1, descs, 1234, 0, None, C.byref(b)) == smppi.ERR_ARG
    assert b.value is None
    assert b"state_kind" in L.smppi_batch_last_error(None)
    p.state_kind = 0           # the same set passes the checks that come before
    assert L.smppi_step_noalloc(C.byref(p), None, None, 0, 0, None, None) == smppi.ERR_ARG
    assert b"NULL" in L.smppi_last_error(None)


def test_wait_timeout_self_test_host_checks(lib):
    """The failure-detection self-test rejects a bad `which` and a NULL status
    word on the host, before any launch."""
    from paper_2302_11719_gb300 import smppi
    smppi.load_library(os.path.join(ROOT, "paper_2302_11719_gb300", "libsmppi.so"))
    L = smppi.load_library()
    assert L.smppi_debug_wait_timeout(2, 1234, None) == smppi.ERR_ARG
    assert b"which" in L.smppi_last_error(None)
    assert L.smppi_debug_wait_timeout(0, None, None) == smppi.ERR_ARG
    assert b"NULL" in L.smppi_last_error(None)


def test_last_error_is_per_thread(lib):
    """A handle-less failure on one host thread does not overwrite the message
    another thread reads."""
    import threading
    from paper_2302_11719_gb300 import smppi
    smppi.load_library(os.path.join(ROOT, "paper_2302_11719_gb300", "libsmppi.so"))
    L = smppi.load_library()
    assert L.smppi_debug_wait_timeout(2, 1234, None) == smppi.ERR_ARG
    other = []

    def worker():
        other.append(L.smppi_debug_wait_timeout(0, None, None))
        other.append(L.smppi_last_error(None))
    th = threading.Thread(target=worker)
    th.start()
    th.join()
    assert other[0] == smppi.ERR_ARG and b"NULL" in other[1]
    assert b"which" in L.smppi_last_error(None)


def test_header_is_plain_c_and_links_from_c(lib, tmp_path):
    """include/smppi.h is a C header (strict C99, no C++ constructs) and a C
    program links against libsmppi.so and calls it; the call here needs no GPU
    (default parameters, then a create that fails its host-side check)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "t.c"
    src.write_text(
        '#include <stdio.h>\n#include "smppi.h"\n'
        "int main(void) {\n"
        "    smppi_params p;\n    smppi_handle* h = 0;\n"
        "    smppi_default_params(&p);\n"
        "    smppi_status s = smppi_create(&p, 0, &h);\n"
        '    printf("%d %d\\n", p.K, (int)s);\n'
        "    return (s == SMPPI_ERR_ARG && h == 0) ? 0 : 1;\n}\n")
    libdir = os.path.join(ROOT, "paper_2302_11719_gb300")
    exe = tmp_path / "t"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lsmppi",
                        "-Wl,-rpath," + libdir, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.split() == ["256", "1"], (r.stdout, r.stderr)
