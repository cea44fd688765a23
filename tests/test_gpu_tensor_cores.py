"""Tensor-core (TF32) multi-RHS subdomain solves against the oracle.

With complex64 factors and 16 or more right-hand sides, the stage solves and
the construction of the boundary operators K run as tcgen05 MMAs with FP32
accumulation (k_tc.cu).  Tolerances, from the arithmetic:
* default (3xTF32): every operand is hi + lo, two TF32 numbers, and the three
  products above roundoff are kept, so each product carries ~2^-21 = 4.8e-7
  relative error (8x the complex64 unit roundoff 6e-8).  The complex64 CUDA-core
  path measures 4e-6..1e-5 against the oracle, an amplification of 60..170 by
  the block recursion over the grid rows, so 3xTF32 should land near
  170 x 4.8e-7 = 8e-5 (measured up to 1.6e-4: the tensor cores' FP32 accumulation
  adds its own rounding).  Bar: 5e-4.
* plain TF32 (tensor_cores="tf32"): u = 2^-11 = 4.9e-4 per operand, expected up
  to 170 x 4.9e-4 = 8e-2, measured ~1.7e-3.  Bar: 6e-3.
The FGMRES solution does not inherit this error: the residual, the Arnoldi
basis and the update stay FP64, so a solve to 1e-9 matches the direct solve to
the same 1e-5 as the complex128 path.

Cases: 1 and 2 tiles of 128 nodes (subdomains 17..131 nodes wide), ragged
RHS blocks (40 = 32 + 8, 70 = 64 + 6), both schedules, with and without the
boundary operators.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W
from oracle import Decomposition, Sweeper, assemble_operator

TF32_PRECOND_TOL = 5e-4      # rel. L2 of one 3xTF32 preconditioner application vs the oracle
PLAIN_TF32_TOL = 6e-3        # the same with plain TF32 operands


@pytest.fixture(scope="module")
def H():
    from paper_2209_10886_gb300 import build
    build.build()
    from paper_2209_10886_gb300 import helm
    helm.lib()
    return helm


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cuda(x, dtype=torch.complex128):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


CASES = {
    "tiny_2x2": lambda: W.workload("tiny"),
    "uneven_4x3": lambda: W.workload("custom", n=70, N1=4, N2=3, medium="layered", seed=4,
                                     xcuts=[0, 17, 35, 52, 70], ycuts=[0, 25, 46, 70]),
    "wide_2x2_131": lambda: W.workload("custom", n=262, N1=2, N2=2, medium="layered", seed=7,
                                       xcuts=[0, 131, 262], ycuts=[0, 129, 262]),
}


def make(H, w, tensor_cores=True, boundary_operators=True, autotune=True, tc_iface_min_ctas=-1):
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts,
                  boundary_operators=boundary_operators, tensor_cores=tensor_cores, autotune=autotune,
                  tc_iface_min_ctas=tc_iface_min_ctas)
    return p.factor("c64")


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("nrhs", [16, 40, 70])
def test_tensor_core_precond_matches_oracle(H, case, nrhs):
    w = CASES[case]()
    p = make(H, w)
    sw = Sweeper(Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts))
    r = W.random_complex((nrhs, w.N), 11)
    z = p.precond_apply(cuda(r), sched="BSP").cpu().numpy()
    for k in sorted({0, 7, 31, 32, nrhs - 1} & set(range(nrhs))):
        e = rel(z[k], sw.precondition(r[k], "BSP"))
        print(f"{case} nrhs {nrhs} TF32 rhs{k}: rel {e:.2e}")
        assert e <= TF32_PRECOND_TOL
    p.close()


@pytest.mark.parametrize("sched", ["BSP", "SP"])
def test_tensor_core_stages_without_boundary_operators(H, sched):
    """Every stage is a full multi-RHS block solve on the tensor cores."""
    w = CASES["uneven_4x3"]()
    p = make(H, w, boundary_operators=False)
    sw = Sweeper(Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts))
    r = W.random_complex((24, w.N), 12)
    z = p.precond_apply(cuda(r), sched=sched).cpu().numpy()
    for k in (0, 23):
        e = rel(z[k], sw.precondition(r[k], sched))
        print(f"uneven_4x3 {sched} TF32 stages rhs{k}: rel {e:.2e}")
        assert e <= TF32_PRECOND_TOL
    p.close()


@pytest.mark.parametrize("case", ["tiny_2x2", "wide_2x2_131"])
def test_plain_tf32_mode(H, case):
    """tensor_cores='tf32': one MMA per product on TF32-rounded operands (64 RHS per CTA
    for 128-node subdomains)."""
    w = CASES[case]()
    p = make(H, w, tensor_cores="tf32")
    sw = Sweeper(Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts))
    r = W.random_complex((70, w.N), 15)
    z = p.precond_apply(cuda(r), sched="BSP").cpu().numpy()
    for k in (0, 63, 64, 69):
        e = rel(z[k], sw.precondition(r[k], "BSP"))
        print(f"{case} plain TF32 rhs{k}: rel {e:.2e}")
        assert e <= PLAIN_TF32_TOL
    p.close()


def test_tensor_core_and_cuda_core_paths_agree_on_few_rhs(H):
    """Below 16 RHS only the construction of K uses the tensor cores."""
    w = CASES["tiny_2x2"]()
    a, b = make(H, w, tensor_cores=True), make(H, w, tensor_cores=False)
    r = cuda(W.random_complex((2, w.N), 13))
    za, zb = a.precond_apply(r).cpu().numpy(), b.precond_apply(r).cpu().numpy()
    e = rel(za, zb)
    print(f"tiny_2x2 TF32 K vs FP32 K, 2 RHS: rel {e:.2e}")
    assert e <= TF32_PRECOND_TOL
    a.close(); b.close()


def test_tensor_core_fgmres_matches_direct_solve(H):
    w = CASES["uneven_4x3"]()
    p = make(H, w)
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    f = W.random_complex((20, w.N), 14)
    u, info, _ = p.solve(cuda(f), tol=1e-9, restart=60, maxit=2000)
    u = u.cpu().numpy()
    lu = spla.splu(A)
    for k in (0, 19):
        ref = lu.solve(w.h ** 2 * f[k])
        rr = np.linalg.norm(w.h ** 2 * f[k] - A @ u[k]) / np.linalg.norm(w.h ** 2 * f[k])
        print(f"uneven_4x3 TF32 FGMRES rhs{k}: iters {info[k][0]}, true relres {rr:.2e}, rel {rel(u[k], ref):.2e}")
        assert info[k][1] <= 1e-9 and rr <= 1.01e-9
        assert rel(u[k], ref) <= 1e-5
    p.close()


def test_interface_krylov_with_tensor_core_stages(H):
    """20 RHS: liftings and reconstructions on the tensor cores, the interface
    problem solved by FGMRES inside the preconditioner."""
    w = CASES["uneven_4x3"]()
    p = make(H, w)
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    f = W.random_complex((20, w.N), 23)
    u, info, _ = p.solve(cuda(f), tol=1e-9, restart=30, maxit=300, inner_maxit=60, inner_tol=1e-3)
    u = u.cpu().numpy()
    lu = spla.splu(A)
    for k in (0, 19):
        ref = lu.solve(w.h ** 2 * f[k])
        print(f"uneven_4x3 TF32 interface Krylov rhs{k}: outer its {info[k][0]}, rel {rel(u[k], ref):.2e}")
        assert info[k][1] <= 1e-9 and rel(u[k], ref) <= 1e-5
    p.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("nrhs", [16, 20, 40, 70])
def test_tensor_core_interface_stages(H, case, nrhs):
    """Interface stages as tcgen05 GEMMs (tc_iface_kernel: 128 output rows x 16 or 32 RHS
    per CTA, boundary points in chunks of 16; ragged RHS blocks 20 = 16 + 4, 40 = 32 + 8,
    70 = 32 + 32 + 6; 1..3 row tiles and ragged chunks) against the CUDA-core stages and
    the oracle.  The fixed rules (no autotuner) pick the tensor cores from 16 RHS; every
    stage takes them here (tc_iface_min_ctas = 1), however few CTAs it makes."""
    w = CASES[case]()
    a = make(H, w, autotune=False, tc_iface_min_ctas=1)
    b = make(H, w, tensor_cores=False, autotune=False)
    assert H.iface_shape(a, nrhs)["tensor_cores"] == 3
    assert H.iface_shape(a, nrhs)["tensor_rhs_per_cta"] == (32 if nrhs >= 32 else 16)
    assert H.iface_shape(b, nrhs)["tensor_cores"] == 0
    assert H.iface_shape(a, 15)["tensor_cores"] == 0
    sw = Sweeper(Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts))
    r = W.random_complex((nrhs, w.N), 31)
    for sched in ("BSP", "SP"):
        za = a.precond_apply(cuda(r), sched=sched).cpu().numpy()
        zb = b.precond_apply(cuda(r), sched=sched).cpu().numpy()
        e_ab = rel(za, zb)
        print(f"{case} nrhs {nrhs} {sched}: tensor-core vs CUDA-core interface stages rel {e_ab:.2e}")
        assert e_ab <= TF32_PRECOND_TOL
        for k in sorted({0, 15, 16, 31, 32, nrhs - 1} & set(range(nrhs))):
            e = rel(za[k], sw.precondition(r[k], sched))
            assert e <= TF32_PRECOND_TOL, (sched, k, e)
    a.close(); b.close()


def test_tensor_core_interface_stages_plain_tf32(H):
    w = CASES["wide_2x2_131"]()
    p = make(H, w, tensor_cores="tf32", autotune=False, tc_iface_min_ctas=1)
    assert H.iface_shape(p, 40)["tensor_cores"] == 1
    sw = Sweeper(Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts))
    r = W.random_complex((40, w.N), 32)
    z = p.precond_apply(cuda(r), sched="BSP").cpu().numpy()
    for k in (0, 31, 32, 39):
        e = rel(z[k], sw.precondition(r[k], "BSP"))
        print(f"wide_2x2_131 plain TF32 interface stages rhs{k}: rel {e:.2e}")
        assert e <= PLAIN_TF32_TOL
    p.close()


def test_interface_krylov_with_tensor_core_interface_stages(H):
    """The interface FGMRES with every interface stage on the tensor cores (fixed rules,
    20 RHS) still converges to the direct solution: the outer FGMRES keeps FP64."""
    w = CASES["uneven_4x3"]()
    p = make(H, w, autotune=False, tc_iface_min_ctas=1)
    assert H.iface_shape(p, 20)["tensor_cores"] == 3
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    f = W.random_complex((20, w.N), 33)
    u, info, _ = p.solve(cuda(f), tol=1e-9, restart=30, maxit=300, inner_maxit=60, inner_tol=1e-3)
    u = u.cpu().numpy()
    lu = spla.splu(A)
    for k in (0, 19):
        ref = lu.solve(w.h ** 2 * f[k])
        print(f"uneven_4x3 tensor-core interface stages, interface Krylov rhs{k}: outer its {info[k][0]}, "
              f"rel {rel(u[k], ref):.2e}")
        assert info[k][1] <= 1e-9 and rel(u[k], ref) <= 1e-5
    p.close()


@pytest.mark.parametrize("case", ["tiny_2x2", "uneven_4x3"])
def test_tensor_core_factorisation_matches_oracle(H, case):
    """precond_factor with the Gauss-Jordan trailing updates on the tensor cores (blocked
    elimination, panels of 16 columns, 3xTF32 updates; subdomains up to 128 nodes wide)
    against the oracle and against the CUDA-core elimination: one BSP application with
    1 and 3 RHS (the CUDA-core block solves, so only the factors differ).  The factors
    carry the 3xTF32 products' 2^-21 instead of FP32's 2^-24: bar as for the tensor-core
    solves."""
    w = CASES[case]()
    mk = lambda tcf: H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts,
                               tc_factor=tcf).factor("c64")
    pt, pc = mk(True), mk(False)
    assert pt.factor_on_tensor_cores() and not pc.factor_on_tensor_cores()
    sw = Sweeper(Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts))
    r = W.random_complex((3, w.N), 17)
    zt = pt.precond_apply(cuda(r)).cpu().numpy()
    zc = pc.precond_apply(cuda(r)).cpu().numpy()
    for k in range(3):
        ref = sw.precondition(r[k], "BSP")
        et, ec = rel(zt[k], ref), rel(zc[k], ref)
        print(f"{case} rhs{k}: tensor-core factors rel {et:.2e}, CUDA-core factors rel {ec:.2e}")
        assert et <= TF32_PRECOND_TOL
    q = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts).factor("c128")
    assert not q.factor_on_tensor_cores()
    pt.close(); pc.close(); q.close()


def test_tensor_core_factorisation_solves_to_the_direct_solution(H):
    w = CASES["uneven_4x3"]()
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts).factor("c64")
    assert p.factor_on_tensor_cores()
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    u, info, _ = p.solve(cuda(w.f), tol=1e-9, restart=30, maxit=300, inner_maxit=60, inner_tol=1e-3)
    ref = spla.spsolve(A, w.h ** 2 * w.f[0])
    e = rel(u.cpu().numpy()[0], ref)
    print(f"tensor-core factors, interface-Krylov solve: its {info[0][0]}, relres {info[0][1]:.2e}, rel {e:.2e}")
    assert info[0][1] <= 1e-9 and e <= 1e-5
    p.close()
