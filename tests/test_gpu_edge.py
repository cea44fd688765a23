"""Edge cases of the C ABI and of the decomposition, on the GPU.

* Empty inputs: nrhs = 0 is a no-op for precond_apply, helm_matvec and
  gmres_solve (HELM_OK, the output untouched).
* Degenerate decompositions: one subdomain (no interfaces: the preconditioner
  is the direct solve, for every transmission condition), subdomains of two to
  four nodes per side, and one column or one row of subdomains with the HABC.
* The widest subdomain the factor layout takes (256 nodes) works; 257 is refused
  with HELM_ERR_ARG before any allocation.
Tolerances as in test_gpu_parity.py: complex128 1e-10 against the oracle.
"""
import ctypes
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W
from oracle import Decomposition, Sweeper, assemble_operator


@pytest.fixture(scope="module")
def H():
    from paper_2209_10886_gb300 import build
    build.build()
    from paper_2209_10886_gb300 import helm
    helm.lib()
    return helm


def cuda(x, dtype=torch.complex128):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_zero_rhs_is_a_noop(H):
    w = W.workload("custom", n=30, N1=2, N2=2, medium="layered", seed=1)
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts).factor("c64")
    L = H.lib()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    z = torch.full((1, w.N), 7.0 + 0j, dtype=torch.complex128, device="cuda")
    r = torch.zeros((1, w.N), dtype=torch.complex128, device="cuda")
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    assert L.precond_apply(p._h, 0, vp(r), vp(z), 0, st) == 0
    assert L.helm_matvec(p._h, vp(r), vp(z), 0, st) == 0
    o = H.default_opts()
    assert L.gmres_solve(p._h, vp(r), vp(z), 0, ctypes.byref(o), None, st) == 0
    torch.cuda.synchronize()
    assert bool(torch.all(z == 7.0))
    p.close()


@pytest.mark.parametrize("transmission", ["optimized", "impedance", "habc"])
@pytest.mark.parametrize("prec,tol", [("c128", 1e-10), ("c64", 1e-4)])
def test_one_subdomain_is_the_direct_solve(H, transmission, prec, tol):
    w = W.workload("custom", n=48, N1=1, N2=1, medium="layered", seed=2)
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), 1, 1, w.xcuts, w.ycuts,
                  transmission=transmission).factor(prec)
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    r = W.random_complex((2, w.N), 70)
    z = p.precond_apply(cuda(r)).cpu().numpy()
    for k in range(2):
        e = rel(z[k], spla.spsolve(A, r[k]))
        print(f"one subdomain, {transmission} {prec}: rel {e:.2e}")
        assert e <= tol
    p.close()


@pytest.mark.parametrize("transmission", ["optimized", "habc"])
def test_tiny_subdomains_match_oracle(H, transmission):
    """3 x 3 subdomains of 3 or 4 nodes per side (interface sides of 3-4 points)."""
    w = W.workload("custom", n=10, N1=3, N2=3, medium="layered", seed=3)
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), 3, 3, w.xcuts, w.ycuts,
                  transmission=transmission).factor("c128")
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts, transmission=transmission)
    sw = Sweeper(dec)
    r = W.random_complex((2, w.N), 71)
    for sched in ("BSP", "SP"):
        z = p.precond_apply(cuda(r), sched=sched).cpu().numpy()
        for k in range(2):
            e = rel(z[k], sw.precondition(r[k], sched))
            print(f"tiny subdomains {transmission} {sched} rhs{k}: rel {e:.2e}")
            assert e <= 1e-10
    p.close()


@pytest.mark.parametrize("N1,N2", [(1, 3), (3, 1)])
def test_habc_on_one_column_or_row_matches_oracle(H, N1, N2):
    w = W.workload("custom", n=40, N1=N1, N2=N2, medium="layered", seed=5)
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), N1, N2, w.xcuts, w.ycuts,
                  transmission="habc").factor("c128")
    sw = Sweeper(Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts, transmission="habc"))
    r = W.random_complex(w.N, 72)
    for sched in ("BSP", "SP"):
        e = rel(p.precond_apply(cuda(r), sched=sched).cpu().numpy(), sw.precondition(r, sched))
        print(f"HABC {N1}x{N2} {sched}: rel {e:.2e}")
        assert e <= 1e-10
    p.close()


def test_subdomain_width_limit(H):
    """256-node subdomains (two tensor-core tiles) factor and apply; 257 is refused."""
    n = 512
    w = W.workload("custom", n=n, N1=2, N2=2, medium="layered", seed=6, xcuts=[0, 256, 512], ycuts=[0, 256, 512])
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), 2, 2, w.xcuts, w.ycuts).factor("c64")
    assert not p.factor_on_tensor_cores()            # the tensor-core elimination takes up to 128 nodes
    z = p.precond_apply(cuda(W.random_complex((1, w.N), 73)))
    assert bool(torch.isfinite(torch.view_as_real(z)).all())
    p.close()
    with pytest.raises(H.HelmError) as e:
        H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), 2, 2, [0, 257, 512], [0, 256, 512])
    assert e.value.status == 1 and "256" in str(e.value)
