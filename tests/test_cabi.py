"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/csk.h declares, and rejects invalid arguments before
touching the device."""
import ctypes
import os
import subprocess

import pytest

from paper_2004_02480_gb300 import csk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(csk.LIB_PATH):
        from paper_2004_02480_gb300 import build
        build.build()
    return csk.lib()


def test_exports_every_declared_function(L):
    names = csk.header_functions()
    assert "csk_solve" in names and "csk_sketch" in names
    out = subprocess.run(["nm", "-D", "--defined-only", csk.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(L, n)


def test_defaults_follow_section3(L):
    p = csk.csk_params_default()
    assert p.tol == 1e-6 and p.max_iter == 20000 and p.d == 0 and p.path == csk.GEMV
    assert L.csk_version() >= 100
    for code in (0, 1, -1, -2, -3, -4, -5, -6):
        assert L.csk_strerror(code).startswith(b"CSK_")


def test_workspace_sizes(L):
    assert L.csk_sketch_workspace_size(0, 5) == 0
    assert L.csk_sketch_workspace_size(10, 0) == 0
    a = L.csk_sketch_workspace_size(1000, 10)
    b = L.csk_sketch_workspace_size(100000, 10)
    assert 0 < a < b and a % 256 == 0
    p = csk.csk_params_default(d=500)
    s1 = csk.csk_solve_workspace_size(2000, 50, csk.CSK_F64, p)
    s2 = csk.csk_solve_workspace_size(2000, 50, csk.CSK_F32, p)
    assert s1 > s2 > 0
    p0 = csk.csk_params_default(d=0)
    assert csk.csk_solve_workspace_size(2000, 50, csk.CSK_F32, p0) > 0
    assert csk.csk_solve_workspace_size(2000, 50, 7, p) == 0


def test_invalid_arguments_rejected_on_host(L):
    fake = ctypes.c_void_p(256)          # never dereferenced: checks come first
    V = ctypes.c_void_p
    # NULL A, m < 1, lda < n, bad dtype, d < 1
    assert L.csk_sketch(None, 10, 2, 2, None, 0, 0, 0, 3, 0, fake, None, None, None, None,
                        fake, 1 << 20, None) == csk.CSK_EINVAL
    assert L.csk_sketch(fake, 0, 2, 2, None, 0, 0, 0, 3, 0, fake, None, None, None, None,
                        fake, 1 << 20, None) == csk.CSK_EINVAL
    assert L.csk_sketch(fake, 10, 4, 2, None, 0, 0, 0, 3, 0, fake, None, None, None, None,
                        fake, 1 << 20, None) == csk.CSK_EINVAL
    assert L.csk_sketch(fake, 10, 2, 2, None, 0, 0, 5, 3, 0, fake, None, None, None, None,
                        fake, 1 << 20, None) == csk.CSK_EINVAL
    assert L.csk_sketch(fake, 10, 2, 2, None, 0, 0, 0, 0, 0, fake, None, None, None, None,
                        fake, 1 << 20, None) == csk.CSK_EINVAL
    # workspace too small / misaligned
    assert L.csk_sketch(fake, 10, 2, 2, None, 0, 0, 0, 3, 0, fake, None, None, None, None,
                        fake, 16, None) == csk.CSK_EINVAL
    assert L.csk_sketch(fake, 10, 2, 2, None, 0, 0, 0, 3, 0, fake, None, None, None, None,
                        V(264), 1 << 20, None) == csk.CSK_EINVAL
    # nrhs > 0 without B
    assert L.csk_sketch(fake, 10, 2, 2, None, 0, 1, 0, 3, 0, fake, fake, None, None, None,
                        fake, 1 << 20, None) == csk.CSK_EINVAL
    # too large for 32-bit row indices
    assert L.csk_sketch(fake, 1 << 32, 2, 2, None, 0, 0, 0, 3, 0, fake, None, None, None,
                        None, fake, 1 << 20, None) == csk.CSK_ENOMEM
    p = csk.csk_params_default(d=3)
    bp = ctypes.byref(p)
    assert L.csk_solve(fake, 10, 2, 2, None, 0, bp, None, None, fake, fake, fake, 1 << 30,
                       None) == csk.CSK_EINVAL
    assert L.csk_solve(fake, 10, 2, 2, fake, 0, None, None, None, fake, fake, fake, 1 << 30,
                       None) == csk.CSK_EINVAL
    assert L.csk_solve(fake, 10, 2, 2, fake, 0, bp, None, None, fake, fake, fake, 8,
                       None) == csk.CSK_EINVAL
    bad = csk.csk_params_default(d=3, tol=-1.0)
    assert L.csk_solve(fake, 10, 2, 2, fake, 0, ctypes.byref(bad), None, None, fake, fake, fake,
                       1 << 30, None) == csk.CSK_EINVAL
    bad = csk.csk_params_default(d=3, ik_log_len=5)
    assert L.csk_solve(fake, 10, 2, 2, fake, 0, ctypes.byref(bad), None, None, fake, fake, fake,
                       1 << 30, None) == csk.CSK_EINVAL
    g = csk.csk_params_default(d=3, path=csk.GRAM)
    assert L.csk_solve(fake, 10, 2, 2, fake, 1, ctypes.byref(g), None, None, fake, fake, fake,
                       1 << 30, None) == csk.CSK_EUNSUPPORTED
    g0 = csk.csk_params_default(d=0, path=csk.GRAM)
    assert L.csk_solve(fake, 10, 2, 2, fake, 0, ctypes.byref(g0), None, None, fake, fake, fake,
                       1 << 30, None) == csk.CSK_EUNSUPPORTED


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        csk.csk_sketch(torch.zeros(4, 2), 2, 0)


def test_host_many_checks_on_host(L):
    """csk_solve_host_many validates every problem before it touches CUDA."""
    import numpy as np
    p = csk.csk_params_default(d=8)
    A = np.zeros((40, 4), np.float32)
    b = np.zeros(40, np.float32)
    out = dict(x_out=np.zeros(5, np.float32), info=np.zeros(1, csk.INFO_DTYPE))
    probs = [csk.HostProblem(A=A, b=b, **out),
             csk.HostProblem(A=np.zeros((60, 5), np.float32), b=np.zeros(60, np.float32), **out)]
    arr, dt = csk._host_problems(probs)
    one = csk.csk_solve_workspace_size(60, 5, csk.CSK_F32, p)
    need = L.csk_solve_host_many_workspace_size(arr, 2, dt, ctypes.byref(p))
    assert need > one > 0
    assert L.csk_solve_host_many_workspace_size(arr, 0, dt, ctypes.byref(p)) == 0
    fake = ctypes.c_void_p(256)
    assert L.csk_solve_host_many(arr, 0, dt, ctypes.byref(p), fake, need, None) == csk.CSK_OK
    assert L.csk_solve_host_many(arr, -1, dt, ctypes.byref(p), fake, need, None) == csk.CSK_EINVAL
    assert L.csk_solve_host_many(arr, 2, dt, ctypes.byref(p), fake, need - 256, None) == csk.CSK_EINVAL
    assert L.csk_solve_host_many(arr, 2, dt, None, fake, need, None) == csk.CSK_EINVAL
    arr[1].lda = 3                                  # lda < n
    assert L.csk_solve_host_many(arr, 2, dt, ctypes.byref(p), fake, need, None) == csk.CSK_EINVAL
    arr[1].lda = 5
    arr[0].b = None
    assert L.csk_solve_host_many(arr, 2, dt, ctypes.byref(p), fake, need, None) == csk.CSK_EINVAL


def test_synth_systems_checks_on_host(L):
    """csk_synth_systems rejects bad sizes before touching CUDA."""
    fake = 256
    ok = csk.csk_synth_system(100, 10, 4, 0, 7, fake, fake, fake)
    arr = (csk.csk_synth_system * 2)(ok, ok)
    assert L.csk_synth_systems(arr, 0, None) == csk.CSK_OK
    assert L.csk_synth_systems(None, 1, None) == csk.CSK_EINVAL
    assert L.csk_synth_systems(arr, -1, None) == csk.CSK_EINVAL
    arr[1] = csk.csk_synth_system(100, 10, 17, 0, 7, fake, fake, fake)    # > 16 right-hand sides
    assert L.csk_synth_systems(arr, 2, None) == csk.CSK_EINVAL
    arr[1] = csk.csk_synth_system(100, 10, 4, 0, 7, None, fake, fake)
    assert L.csk_synth_systems(arr, 2, None) == csk.CSK_EINVAL
    arr[1] = csk.csk_synth_system(0, 10, 4, 0, 7, fake, fake, fake)
    assert L.csk_synth_systems(arr, 2, None) == csk.CSK_EINVAL


def test_info_sync_and_workspace_size_checks(L):
    """csk_info_sync rejects NULL records before any CUDA call;
    csk_workspace_size covers csk_sketch, csk_solve and the one-system
    batched solve of the same shape, and is 0 for invalid sizes."""
    fake = ctypes.c_void_p(256)
    assert L.csk_info_sync(None, fake, None) == csk.CSK_EINVAL
    assert L.csk_info_sync(fake, None, None) == csk.CSK_EINVAL
    m, n, d = 100000, 500, 5000
    for dt in (csk.CSK_F32, csk.CSK_F64):
        for path in (csk.GEMV, csk.AUTO) + ((csk.GRAM,) if dt == csk.CSK_F32 else ()):
            w = L.csk_workspace_size(m, n, d, 1, dt, path)
            p = csk.csk_params_default(d=d, path=path)
            assert w >= csk.csk_solve_workspace_size(m, n, dt, p) > 0
            assert w >= L.csk_sketch_workspace_size(m, d) > 0
    one = csk.csk_system(256, m, n, n, 256, 4, 4, 0, d, 0, None, None, 256, 256)
    arr = (csk.csk_system * 1)(one)
    assert L.csk_workspace_size(m, n, d, 4, csk.CSK_F32, csk.GRAM) >= \
        L.csk_solve_batched_workspace_size(arr, 1) > 0
    assert L.csk_workspace_size(m, n, 0, 1, csk.CSK_F32, csk.GEMV) == \
        csk.csk_solve_workspace_size(m, n, csk.CSK_F32, csk.csk_params_default(d=0))
    for bad in ((0, n, d, 1, 0, 0), (m, 0, d, 1, 0, 0), (m, n, -1, 1, 0, 0), (m, n, d, -1, 0, 0),
                (m, n, d, 1, 5, 0), (m, n, d, 1, 0, 7)):
        assert L.csk_workspace_size(*bad) == 0


def test_exchange_floor_checks_on_host(L):
    fake = ctypes.c_void_p(256)
    assert L.csk_exchange_floor_workspace_size(0) == 0
    assert L.csk_exchange_floor_workspace_size(321) == 0
    need = L.csk_exchange_floor_workspace_size(91)
    assert need >= 2 * 91 * 91 * 32 and need % 256 == 0
    assert L.csk_exchange_floor(0, 10, fake, need, None) == csk.CSK_EINVAL
    assert L.csk_exchange_floor(91, 0, fake, need, None) == csk.CSK_EINVAL
    assert L.csk_exchange_floor(91, 10, None, need, None) == csk.CSK_EINVAL
    assert L.csk_exchange_floor(91, 10, fake, need - 256, None) == csk.CSK_EINVAL
    assert L.csk_exchange_floor(91, 10, ctypes.c_void_p(264), need, None) == csk.CSK_EINVAL


def test_batched_log_arguments_checked_on_host(L):
    """The per-step logs of csk_solve_batched name one (system, right-hand
    side) pair of the caller's array; out-of-range pairs and a log length
    without a buffer are rejected before any CUDA call."""
    one = csk.csk_system(256, 1000, 10, 10, 256, 2, 2, 0, 100, 0, None, None, 256, 256)
    arr = (csk.csk_system * 1)(one)
    fake = ctypes.c_void_p(256)
    for kw in (dict(ik_log=256, ik_log_len=5, log_system=1), dict(ik_log=256, ik_log_len=5, log_rhs=2),
               dict(ik_log_len=5), dict(x_log_len=5), dict(x_log=256, x_log_len=5, log_system=-1)):
        p = csk.csk_params_default(**kw)
        assert L.csk_solve_batched(arr, 1, ctypes.byref(p), fake, 1 << 40, None) == csk.CSK_EINVAL
