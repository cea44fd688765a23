"""Failure paths of the library, made to happen without faulting the GPU.

* A bounded device wait that gives up: helm_opts.wait_cycles sets how long the
  grid barriers of the Gram-Schmidt kernels wait; with one cycle every barrier
  that is not passed at once gives up.  The kernels that wait there hold no bulk
  copy or MMA in flight (the fused classical Gram-Schmidt step of the interface
  and of the volume iterations), so they record HELM_ERR_TIMEOUT in the device
  status word and return.  The call must report HELM_ERR_TIMEOUT with a message;
  after precond_factor the same handle must solve normally again.
* The device budget: a handle whose factors would exceed helm_setup_opts
  .device_budget gets HELM_ERR_OOM from precond_factor (nothing allocated); one
  whose factors fit but whose Krylov workspace does not gets HELM_ERR_OOM from
  gmres_solve.
* Non-convergence: maxit = 1 at a tolerance one step cannot reach gives
  HELM_ERR_NO_CONVERGENCE with a message, the last iterate in u and the info
  entries filled (one step, the true relative residual of that iterate).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W
from oracle import assemble_operator


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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def uneven():
    return W.workload("custom", n=70, N1=4, N2=3, medium="layered", seed=4, xcuts=[0, 17, 35, 52, 70],
                      ycuts=[0, 25, 46, 70])


@pytest.mark.parametrize("where", ["interface", "volume"])
def test_expired_wait_reports_timeout_and_the_handle_recovers(H, where):
    w = uneven()
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts).factor("c64")
    f = cuda(w.f)
    kw = dict(tol=1e-9, restart=30, maxit=300)
    if where == "interface":
        kw.update(inner_maxit=60, inner_tol=1e-3)       # the interface iterations' fused CGS2 step
    else:
        kw.update(ortho="cgs2")                         # the volume iterations' fused CGS2 step
    with pytest.raises(H.HelmError) as e:
        p.solve(f, wait_cycles=1, **kw)
    assert e.value.status == 6 and "timed out" in str(e.value)
    # the status word was read and cleared; a new factorisation makes the handle usable again
    p.factor("c64")
    u, info, _ = p.solve(f, **kw)
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    ref = spla.spsolve(A, w.h ** 2 * w.f[0])
    print(f"{where}: after the timeout, its {info[0][0]}, relres {info[0][1]:.2e}, "
          f"rel {rel(u.cpu().numpy()[0], ref):.2e}")
    assert info[0][1] <= 1e-9 and rel(u.cpu().numpy()[0], ref) <= 1e-5
    p.close()


def test_device_budget_gives_oom(H):
    w = uneven()
    m2 = cuda(w.m2, torch.float64)
    small = H.Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, device_budget=4096)
    with pytest.raises(H.HelmError) as e:
        small.factor("c64")
    assert e.value.status == 3 and "budget" in str(e.value)
    with pytest.raises(H.HelmError) as e:          # still unfactored: nothing was kept
        small.precond_apply(cuda(w.f))
    assert e.value.status == 4
    small.close()
    # the factors (and the boundary operators, about as large here; no tensor-core copy) fit;
    # one RHS's Krylov workspace (2 x 150 + 1 fields of 70^2 complex128, 23.6 MB) does not
    probe = H.Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, tensor_cores=False).factor("c64")
    fb = probe.info()["factor_bytes"]
    probe.close()
    tight = H.Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, tensor_cores=False,
                      device_budget=4 * fb + (1 << 20))
    tight.factor("c64")
    with pytest.raises(H.HelmError) as e:
        tight.solve(cuda(w.f), restart=150)
    assert e.value.status == 3 and "budget" in str(e.value)
    u, info, _ = tight.solve(cuda(w.f), restart=2, maxit=4, raise_on_noconv=False)   # a small workspace fits
    assert info[0][0] == 4
    tight.close()


@pytest.mark.parametrize("inner_maxit", [0, 60])
def test_non_convergence_reports_status_and_fills_info(H, inner_maxit):
    w = uneven()
    A = assemble_operator(w.n, w.h, w.omega, w.m2)
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts).factor("c64")
    fh = W.random_complex((2, w.N), 90)
    f = cuda(fh)
    kw = dict(tol=1e-12, restart=30, maxit=1, inner_maxit=inner_maxit, inner_tol=1e-2)
    with pytest.raises(H.HelmError) as e:
        p.solve(f, **kw)
    assert e.value.status == 5 and "maxit" in str(e.value)
    u, info, _ = p.solve(f, raise_on_noconv=False, **kw)
    u = u.cpu().numpy()
    for k in range(2):
        b = w.h ** 2 * fh[k]
        rr = float(np.linalg.norm(b - A @ u[k]) / np.linalg.norm(b))
        print(f"inner_maxit {inner_maxit} rhs{k}: its {info[k][0]}, relres {info[k][1]:.3e}, host {rr:.3e}")
        assert info[k][0] == 1
        assert 1e-12 < info[k][1] < 1.0          # one minimal-residual step from u = 0
        assert abs(info[k][1] - rr) <= 1e-6 * rr  # the reported residual is that of u
    # the handle is unaffected: the same solve to a reachable tolerance converges
    u2, info2, _ = p.solve(f, tol=1e-9, restart=30, maxit=200, inner_maxit=inner_maxit, inner_tol=1e-2)
    u2 = u2.cpu().numpy()
    for k in range(2):
        b = w.h ** 2 * fh[k]
        assert info2[k][1] <= 1e-9
        assert np.linalg.norm(b - A @ u2[k]) <= 2e-9 * np.linalg.norm(b)
    p.close()
