"""precond_apply_noalloc: the preconditioner for callers that must not allocate.

Some callers cannot allocate device memory while they solve (a memory budget
fixed before the solve phase, or a framework whose caching allocator owns all
device memory).  precond_apply allocates its workspace on first use, so the
library also offers precond_apply_noalloc, which takes its scratch from one
fixed array that is part of the library image.  This file checks, through the
C ABI, that it returns what precond_apply returns, on two calls in a row (the
second call finds the first call's leftovers in the shared array), and that a
request larger than the array is refused before any launch.  It is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W


@pytest.fixture(scope="module")
def H():
    from paper_2209_10886_gb300 import build
    build.build()
    from paper_2209_10886_gb300 import helm
    L = helm.lib()
    L.precond_apply_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p]
    L.precond_apply_noalloc.restype = ctypes.c_int
    return helm


def _noalloc(H, p, r, sched):
    z = torch.empty_like(r)
    st = H.lib().precond_apply_noalloc(p._h, H.SCHED[sched], ctypes.c_void_p(r.data_ptr()),
                                       ctypes.c_void_p(z.data_ptr()), r.numel() // p.N,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, z


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


# the tolerances of the parity tests: complex128 1e-10, complex64 3e-5
@pytest.mark.parametrize("prec,tol", [("c128", 1e-10), ("c64", 3e-5)])
@pytest.mark.parametrize("sched", ["BSP", "SP"])
def test_noalloc_matches_precond_apply_on_two_calls(H, prec, tol, sched):
    w = W.workload("custom", n=60, N1=3, N2=2, medium="layered", seed=3, xcuts=[0, 21, 39, 60], ycuts=[0, 33, 60])
    m2 = torch.as_tensor(w.m2, dtype=torch.float64, device="cuda")
    p = H.Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts).factor(prec)
    for call, nrhs in enumerate((3, 1)):
        r = torch.as_tensor(W.random_complex((nrhs, w.N), 40 + call), device="cuda")
        st, z = _noalloc(H, p, r, sched)
        assert st == 0, H.lib().helm_last_error()
        ref = p.precond_apply(r, sched=sched)
        torch.cuda.synchronize()
        for k in range(nrhs):
            assert _rel(z[k], ref[k]) <= tol
    p.close()


def test_noalloc_refuses_requests_beyond_its_array(H):
    w = W.workload("tiny")
    m2 = torch.as_tensor(w.m2, dtype=torch.float64, device="cuda")
    p = H.Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts).factor("c128")
    nrhs = 200                   # 200 x 16,129 unknowns x 16 B of workspace alone exceed 32 MiB
    r = torch.zeros((nrhs, w.N), dtype=torch.complex128, device="cuda")
    st, _ = _noalloc(H, p, r, "BSP")
    assert st == 1
    assert b"bytes" in H.lib().helm_last_error()
    st, _ = _noalloc(H, p, r[:2], "BSP")       # a fitting request still works afterwards
    assert st == 0
    p.close()


@pytest.mark.parametrize("sched", ["BSP", "SP"])
def test_noalloc_tensor_core_branch_matches_precond_apply(H, sched):
    """Complex64 factors with 16 and 32 RHS: the stages run on the tensor cores, whose
    extra scratch (interface data and boundary values of every subdomain, the scaled
    source in complex64) the call carves from the end of the fixed array.  Without the
    autotuner both entry points take the same fixed launch shapes."""
    w = W.workload("custom", n=60, N1=3, N2=2, medium="layered", seed=3, xcuts=[0, 21, 39, 60], ycuts=[0, 33, 60])
    m2 = torch.as_tensor(w.m2, dtype=torch.float64, device="cuda")
    p = H.Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, autotune=False).factor("c64")
    for call, nrhs in enumerate((16, 32, 16)):
        assert H.iface_shape(p, nrhs)["tensor_cores"] == 3
        r = torch.as_tensor(W.random_complex((nrhs, w.N), 60 + call), device="cuda")
        st, z = _noalloc(H, p, r, sched)
        assert st == 0, H.lib().helm_last_error()
        ref = p.precond_apply(r, sched=sched)
        torch.cuda.synchronize()
        for k in (0, 15, nrhs - 1):
            assert _rel(z[k], ref[k]) <= 3e-5
    p.close()


def test_noalloc_allocates_no_device_memory(H):
    """On a freshly factored problem that never ran precond_apply, calls with growing RHS
    counts (which make precond_apply allocate a larger workspace) leave the device's free
    memory unchanged.  A first problem loads the library's kernels and the fixed array."""
    w = W.workload("custom", n=60, N1=3, N2=2, medium="layered", seed=3, xcuts=[0, 21, 39, 60], ycuts=[0, 33, 60])
    m2 = torch.as_tensor(w.m2, dtype=torch.float64, device="cuda")
    counts = (1, 2, 4, 8, 16)
    rs = [torch.as_tensor(W.random_complex((n, w.N), 80 + n), device="cuda") for n in counts]
    warm = H.Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, autotune=False).factor("c64")
    for r in rs:
        st, _ = _noalloc(H, warm, r, "BSP")
        assert st == 0, H.lib().helm_last_error()
    torch.cuda.synchronize()
    warm.close()
    p = H.Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, autotune=False).factor("c64")
    zs = [torch.empty_like(r) for r in rs]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for r, z in zip(rs, zs):
        st = H.lib().precond_apply_noalloc(p._h, H.SCHED["BSP"], ctypes.c_void_p(r.data_ptr()),
                                           ctypes.c_void_p(z.data_ptr()), r.numel() // p.N,
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, H.lib().helm_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    for r, z in zip(rs, zs):                       # and the results are the preconditioner's
        ref = p.precond_apply(r)
        torch.cuda.synchronize()
        assert _rel(z, ref) <= 3e-5
    p.close()


@pytest.mark.parametrize("prec,tol", [("c128", 1e-10), ("c64", 3e-5)])
def test_noalloc_with_the_habc_transmission(H, prec, tol):
    """The HABC transmission keeps a fourth interface buffer (the liftings' boundary
    values) in the fixed array; two calls in a row against precond_apply."""
    w = W.workload("custom", n=60, N1=3, N2=2, medium="layered", seed=3, xcuts=[0, 21, 39, 60], ycuts=[0, 33, 60])
    m2 = torch.as_tensor(w.m2, dtype=torch.float64, device="cuda")
    p = H.Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, transmission="habc",
                  autotune=False).factor(prec)
    for call, nrhs in enumerate((3, 1)):
        r = torch.as_tensor(W.random_complex((nrhs, w.N), 90 + call), device="cuda")
        st, z = _noalloc(H, p, r, "BSP")
        assert st == 0, H.lib().helm_last_error()
        ref = p.precond_apply(r)
        torch.cuda.synchronize()
        for k in range(nrhs):
            assert _rel(z[k], ref[k]) <= tol
    p.close()
