"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (written per test):
* complex128 path vs oracle: both compute the same operator in FP64 with
  different elimination orders (block-tridiagonal Gauss-Jordan vs sparse LU);
  the difference is roundoff times the local condition number (measured
  2e-15..2e-14 on the field and on the interface nodes); one application <= 1e-12.
* complex64 preconditioner vs the complex128 oracle: unit roundoff 6e-8
  amplified by the block recursion over the grid rows (measured 2e-6..7e-6 on the
  field and up to 1.4e-5 on the interface nodes for subdomains of at most 64 rows,
  2.9e-5 / 3.2e-5 for 131-row ones: an amplification of 30..500; printed with -s).
  Bars per case (C64_BARS) about 3x the measurement; 1e-4 where a test combines
  other paths.
* Every preconditioner comparison also takes the largest error on the interface
  boundary nodes (iface_err) relative to the largest value there.
* Solutions: both sides solve to a true relative residual of 1e-9, so they
  agree to cond(A) * 1e-9; the bar is rel. L2 <= 1e-5.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W
from oracle import Decomposition, Sweeper, assemble_operator
from oracle.adjoint import misfit_gradient_direct

C64_TOL = 1e-4       # rel. L2 of one complex64 preconditioner application vs the oracle
# (field, interface nodes) bars of one complex64 BSP application per case: subdomains of
# at most 64 rows / 131 rows (the block recursion's amplification grows with the rows)
C64_BARS = {"tiny_2x2": (2e-5, 5e-5), "uneven_4x3": (2e-5, 5e-5), "wide_2x2_131": (1e-4, 1e-4)}
C128_BAR = 1e-12


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


def make(H, w, prec="c128", transmission="optimized"):
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts,
                  transmission=transmission)
    p.factor(prec)
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts, transmission=transmission)
    return p, dec


CASES = {
    "tiny_2x2": lambda: W.workload("tiny"),
    "ragged_3x2": lambda: W.workload("custom", n=60, N1=3, N2=2, medium="layered", seed=3,
                                     xcuts=[0, 21, 39, 60], ycuts=[0, 33, 60]),
    "uneven_4x3": lambda: W.workload("custom", n=70, N1=4, N2=3, medium="layered", seed=4,
                                     xcuts=[0, 17, 35, 52, 70], ycuts=[0, 25, 46, 70]),
    "column_1x3": lambda: W.workload("custom", n=40, N1=1, N2=3, medium="layered", seed=5),
    "row_3x1": lambda: W.workload("custom", n=40, N1=3, N2=1, medium="layered", seed=6),
    "wide_2x2_131": lambda: W.workload("custom", n=262, N1=2, N2=2, medium="layered", seed=7,
                                       xcuts=[0, 131, 262], ycuts=[0, 129, 262]),
}


def iface_mask(w):
    """The subdomains' interface boundary nodes (every node next to a cut): the values
    the transmission epilogues form, checked on their own so that an error confined to
    them cannot hide in the norm over the whole field."""
    mask = np.zeros((w.n, w.n), dtype=bool)
    for c in w.xcuts[1:-1]:
        mask[:, c - 1] = mask[:, c] = True
    for c in w.ycuts[1:-1]:
        mask[c - 1, :] = mask[c, :] = True
    return mask.reshape(-1)


def iface_err(z, ref, mask):
    """Largest error on the interface nodes relative to the largest value there."""
    return float(np.abs(z[mask] - ref[mask]).max() / np.abs(ref[mask]).max())


def test_matvec_matches_sparse_matrix(H):
    for name in ("tiny_2x2", "uneven_4x3"):
        w = CASES[name]()
        p, _ = make(H, w)
        A = assemble_operator(w.n, w.h, w.omega, w.m2)
        u = W.random_complex((3, w.N), 1)
        Au = p.matvec(cuda(u)).cpu().numpy()
        ref = np.stack([A @ u[k] for k in range(3)])
        assert np.abs(Au - ref).max() <= 1e-14 * np.abs(ref).max()
        p.close()


@pytest.mark.parametrize("prec,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_single_subdomain_is_direct_solve(H, prec, tol):
    """One subdomain: the preconditioner is the direct solve (measured c128 8e-15,
    c64 2.5e-6 on 75 rows)."""
    w = W.workload("custom", n=75, N1=1, N2=1, medium="layered", seed=2)
    p, _ = make(H, w, prec)
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    r = W.random_complex((2, w.N), 3)
    z = p.precond_apply(cuda(r)).cpu().numpy()
    for k in range(2):
        e = rel(z[k], spla.spsolve(A, r[k]))
        print(f"single subdomain {prec}: rel {e:.2e}")
        assert e <= tol
    p.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("sched", ["BSP", "SP"])
def test_precond_apply_c128_matches_oracle(H, case, sched):
    w = CASES[case]()
    p, dec = make(H, w, "c128")
    sw = Sweeper(dec)
    nrhs = 3 if case in ("tiny_2x2", "uneven_4x3") else 1
    r = W.random_complex((nrhs, w.N), 5)
    z = p.precond_apply(cuda(r), sched=sched).cpu().numpy()
    mask = iface_mask(w)
    for k in range(nrhs):
        ref = sw.precondition(r[k], sched)
        e = rel(z[k], ref)
        ei = iface_err(z[k], ref, mask) if mask.any() else 0.0
        print(f"{case} {sched} c128 rhs{k}: rel {e:.2e}, interface nodes max {ei:.2e}")
        assert e <= C128_BAR and ei <= C128_BAR
    p.close()


@pytest.mark.parametrize("case", ["tiny_2x2", "uneven_4x3", "wide_2x2_131"])
def test_precond_apply_c64_matches_oracle(H, case):
    w = CASES[case]()
    p, dec = make(H, w, "c64")
    sw = Sweeper(dec)
    r = W.random_complex((5, w.N), 6)      # 5 RHS: one CTA of 4 and a ragged CTA of 1
    z = p.precond_apply(cuda(r), sched="BSP").cpu().numpy()
    mask = iface_mask(w)
    for k in range(5):
        ref = sw.precondition(r[k], "BSP")
        e, ei = rel(z[k], ref), iface_err(z[k], ref, mask)
        print(f"{case} BSP c64 rhs{k}: rel {e:.2e}, interface nodes max {ei:.2e}")
        bar_field, bar_iface = C64_BARS[case]
        assert e <= bar_field and ei <= bar_iface
    p.close()


@pytest.mark.parametrize("prec,tol", [("c128", 1e-10), ("c64", C64_TOL)])
def test_without_boundary_operators_matches_oracle(H, prec, tol):
    """Sweep steps as full block-tridiagonal solves (no K): the same operator."""
    w = CASES["uneven_4x3"]()
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts,
                  boundary_operators=False).factor(prec)
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts)
    r = W.random_complex((2, w.N), 9)
    for sched in ("BSP", "SP"):
        z = p.precond_apply(cuda(r), sched=sched).cpu().numpy()
        for k in range(2):
            assert rel(z[k], Sweeper(dec).precondition(r[k], sched)) <= tol
    p.close()


@pytest.mark.parametrize("ortho", [0, 1, 2])
def test_gram_schmidt_variants_agree(H, ortho):
    """Modified (persistent kernel) and reorthogonalised classical Gram-Schmidt
    (fused into one launch per step, and split into reduction kernels) all reach
    the direct solution."""
    import ctypes
    w = CASES["tiny_2x2"]()
    p, _ = make(H, w, "c64")
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    ref = spla.spsolve(A, w.h ** 2 * w.f[0])
    f = cuda(w.f)
    u = torch.empty_like(f)
    o = H.default_opts(restart=40, maxit=500, tol=1e-9, ortho=ortho)
    info = (H.HelmInfo * 1)()
    st = H.lib().gmres_solve(p._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1, ctypes.byref(o),
                             info, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0 and info[0].relres <= 1e-9
    assert rel(u.cpu().numpy()[0], ref) <= 1e-5
    p.close()


@pytest.mark.parametrize("where", ["volume", "interface", "interface_c64"])
def test_fused_cgs2_matches_split(H, where):
    """The fused Arnoldi step (CGS2, norm, normalisation and Givens update in one
    cooperative launch) against the same arithmetic as separate kernels: three RHS
    that converge at different steps (the active flags), both reach the direct
    solution and take the same number of outer steps up to one (two with complex64
    interface vectors, whose FP32 sums round differently in the two forms)."""
    w = CASES["ragged_3x2"]()
    p, _ = make(H, w, "c64" if where == "interface_c64" else "c128")
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    f = W.random_complex((3, w.N), 31)
    f[1, : w.N // 2] = 0.0            # a source in half of the domain
    f[2] = 0.0
    f[2, w.N // 2] = 1.0              # a point source
    kw = dict(tol=1e-9, restart=25, maxit=600)
    if where == "interface":
        kw.update(inner_maxit=80, inner_restart=12, inner_tol=1e-6)
    if where == "interface_c64":
        kw.update(inner_maxit=80, inner_restart=12, inner_tol=1e-4)
    res = {}
    for ortho in ("cgs2", "cgs2_split"):
        u, info, _ = p.solve(cuda(f), ortho=ortho, **kw)
        res[ortho] = (u.cpu().numpy(), info)
    lu = spla.splu(A.tocsc())
    for k in range(3):
        ref = lu.solve(w.h ** 2 * f[k])
        for ortho, (u, info) in res.items():
            print(f"{where} {ortho} rhs{k}: its {info[k][0]}, relres {info[k][1]:.2e}, rel {rel(u[k], ref):.2e}")
            assert info[k][1] <= 1e-9 and rel(u[k], ref) <= 1e-5
        assert abs(res["cgs2"][1][k][0] - res["cgs2_split"][1][k][0]) <= (2 if where == "interface_c64" else 1)
    p.close()


@pytest.mark.parametrize("case", ["ragged_3x2", "uneven_4x3"])
def test_nonoverlapping_bands_match_oracle(H, case):
    """BSP with bands of N1 diagonals that share none (the comparison variant of the
    band rule) against the oracle's BSP with overlap=False, complex128."""
    w = CASES[case]()
    p, dec = make(H, w, "c128")
    r = W.random_complex((2, w.N), 52)
    z = p.precond_apply(cuda(r), sched="BSP_NONOVERLAP").cpu().numpy()
    sw = Sweeper(dec)
    for k in range(2):
        ref = sw.precondition(r[k], "BSP", overlap=False)
        other = sw.precondition(r[k], "BSP", overlap=True)
        e = rel(z[k], ref)
        print(f"{case} BSP non-overlapping rhs{k}: rel {e:.2e} (vs overlapping bands {rel(z[k], other):.2e})")
        assert e <= 1e-10 and rel(z[k], other) > 1e-6
    p.close()


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_autotuned_interface_shape(H, prec):
    """The first application with several RHS times the interface-stage launch shapes
    and keeps the fastest; the result equals the fixed-rule shape's up to the rounding
    of the GEMV sums (their order depends on the RHS per block) or, with complex64
    factors, that of the 3xTF32 tensor-core form the fixed rules pick at 20 RHS."""
    w = CASES["uneven_4x3"]()
    mk = lambda tune: H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts,
                                autotune=tune).factor(prec)
    pa, pb = mk(True), mk(False)
    r = cuda(W.random_complex((20, w.N), 51))
    za = pa.precond_apply(r).cpu().numpy()
    zb = pb.precond_apply(r).cpu().numpy()
    sa, sb = H.iface_shape(pa, 20), H.iface_shape(pb, 20)
    print(prec, "tuned", sa, "fixed", sb, "rel", rel(za, zb))
    assert sa["tuned"] and not sb["tuned"]
    # fixed rules at 20 RHS: blocks of 4 RHS on the CUDA cores, and with complex64 factors
    # the tensor-core form (16 RHS per CTA) for stages of at least two CTAs per SM (none
    # on this small problem)
    if prec == "c64":
        assert sb["tensor_cores"] == 3 and sb["tensor_rhs_per_cta"] == 16 and sb["rhs_per_block"] == 4
    else:
        assert sb["tensor_cores"] == 0 and sb["rhs_per_block"] == 4
    assert not H.iface_shape(pa, 1)["tuned"]
    assert rel(za, zb) <= (1e-5 if prec == "c64" else 1e-12)
    pa.close(); pb.close()


@pytest.mark.parametrize("prec,nrhs", [("c64", 1), ("c128", 1), ("c64", 40), ("c128", 3)])
def test_autotuned_stage_shape(H, prec, nrhs):
    """The first application per RHS count also times the full-stage kernels' launch
    shapes on the liftings (CTAs per subdomain and factor chunk on the CUDA cores; RHS
    per CTA in the tensor-core form) and keeps the fastest: the same solves, so the same
    z up to the rounding of the order of the sums."""
    w = CASES["uneven_4x3"]()
    mk = lambda tune: H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts,
                                autotune=tune).factor(prec)
    pa, pb = mk(True), mk(False)
    r = cuda(W.random_complex((nrhs, w.N), 53))
    za = pa.precond_apply(r).cpu().numpy()
    zb = pb.precond_apply(r).cpu().numpy()
    sa, sb = H.stage_shape(pa, nrhs), H.stage_shape(pb, nrhs)
    print(prec, nrhs, "tuned", sa, "fixed", sb, "rel", rel(za, zb))
    assert sa["tuned"] and not sb["tuned"]
    assert (sa["tensor_rhs_per_cta"] > 0) == (prec == "c64" and nrhs >= 16)
    assert rel(za, zb) <= (C64_TOL if prec == "c64" else 1e-12)
    pa.close(); pb.close()


def test_impedance_transmission_matches_oracle(H):
    w = CASES["ragged_3x2"]()
    p, dec = make(H, w, "c128", transmission="impedance")
    r = W.random_complex(w.N, 8)
    z = p.precond_apply(cuda(r)).cpu().numpy()
    assert rel(z, Sweeper(dec).precondition(r, "BSP")) <= 1e-10
    p.close()


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("sched", ["BSP", "SP"])
def test_gmres_matches_direct_solve(H, prec, sched):
    w = CASES["tiny_2x2"]()
    p, _ = make(H, w, prec)
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    ref = spla.spsolve(A, w.h ** 2 * w.f[0])
    u, info, _ = p.solve(cuda(w.f), tol=1e-9, restart=50, sched=sched)
    u = u.cpu().numpy()[0]
    true_rr = np.linalg.norm(w.h ** 2 * w.f[0] - A @ u) / np.linalg.norm(w.h ** 2 * w.f[0])
    print(f"gmres {prec} {sched}: iters {info[0][0]} relres {info[0][1]:.2e} true {true_rr:.2e} err {rel(u, ref):.2e}")
    assert info[0][1] <= 1e-9 and true_rr <= 1.01e-9
    assert rel(u, ref) <= 1e-5


def test_gmres_multi_rhs_and_initial_guess(H):
    w = W.workload("custom", n=60, N1=3, N2=2, medium="layered", seed=3, nrhs=3,
                   xcuts=[0, 21, 39, 60], ycuts=[0, 33, 60])
    p, _ = make(H, w, "c64")
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    u, info, hist = p.solve(cuda(w.f), tol=1e-9, history=True)
    u = u.cpu().numpy()
    for k in range(3):
        ref = spla.spsolve(A, w.h ** 2 * w.f[k])
        assert rel(u[k], ref) <= 1e-5 and info[k][1] <= 1e-9
        assert len(hist[k]) == info[k][0] and hist[k][-1] <= 1e-9 * 1.0001
    # restarting from the solution needs no iteration
    u2, info2, _ = p.solve(cuda(w.f), x0=cuda(u), tol=1e-9)
    assert all(it == 0 for it, _ in info2)


@pytest.mark.parametrize("prec", ["c128", "c64", "c64_fp64_interface"])
@pytest.mark.parametrize("sched", ["BSP", "SP"])
def test_interface_krylov_gmres_matches_direct_solve(H, prec, sched):
    """inner_maxit > 0: the preconditioner solves the interface problem (I - S) g = b by
    FGMRES with the sweep as its preconditioner (the paper's formulation); the outer
    FP64 FGMRES on the volume still reaches the true residual and the direct solution.
    With complex64 factors the interface vectors are complex64 unless inner_fp64."""
    w = CASES["uneven_4x3"]()
    p, _ = make(H, w, prec.split("_")[0])
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    f = W.random_complex((2, w.N), 22)
    s0 = H.inner_steps(p)
    u, info, _ = p.solve(cuda(f), tol=1e-9, restart=30, maxit=200, sched=sched, inner_maxit=60, inner_tol=1e-3,
                         inner_fp64=prec.endswith("fp64_interface"))
    steps = H.inner_steps(p) - s0
    u = u.cpu().numpy()
    lu = spla.splu(A)
    for k in range(2):
        ref = lu.solve(w.h ** 2 * f[k])
        rr = np.linalg.norm(w.h ** 2 * f[k] - A @ u[k]) / np.linalg.norm(w.h ** 2 * f[k])
        print(f"uneven_4x3 {prec} {sched} interface Krylov rhs{k}: outer its {info[k][0]}, inner steps {steps}, "
              f"true relres {rr:.2e}, rel {rel(u[k], ref):.2e}")
        assert info[k][1] <= 1e-9 and rr <= 1.01e-9
        assert rel(u[k], ref) <= 1e-5
        assert info[k][0] <= 12                     # a few outer steps: the inner solve does the work
    assert steps > 0
    p.close()


@pytest.mark.parametrize("prec", ["c64", "c128", "c64_fp64_interface"])
def test_device_driven_interface_loop_matches_host_loop(H, prec):
    """The interface Arnoldi steps run as a conditional CUDA graph (device-side loop
    control) unless per-launch profiling is on, which takes the host-driven loop; the
    kernels and their order are the same, so are the iterates.  Both schedules on the
    same problem, one after the other (each has its own graph); three RHS that stop at
    different steps (one zero RHS)."""
    w = CASES["uneven_4x3"]()
    p, _ = make(H, w, prec.split("_")[0])
    f = W.random_complex((3, w.N), 41)
    f[1, : w.N // 3] = 0.0
    f[2] = 0.0
    res = {}
    for prof in (False, True):
        H.profile(p, prof)
        for sched in ("BSP", "SP"):
            kw = dict(tol=1e-9, restart=30, maxit=200, sched=sched, inner_maxit=60, inner_restart=12,
                      inner_tol=1e-3, inner_fp64=prec.endswith("fp64_interface"))
            s0 = H.inner_steps(p)
            u, info, _ = p.solve(cuda(f), **kw)
            res[(prof, sched)] = (u.cpu().numpy(), [i[0] for i in info], H.inner_steps(p) - s0)
    H.profile(p, False)
    for sched in ("BSP", "SP"):
        (u0, i0, n0), (u1, i1, n1) = res[(False, sched)], res[(True, sched)]
        print(f"{prec} {sched}: device loop its {i0} inner {n0}, host loop its {i1} inner {n1}")
        assert i0 == i1 and n0 == n1
        assert np.all(u0[2] == 0) and i0[2] == 0
        assert rel(u0[:2], u1[:2]) <= 1e-12
    # the schedules differ (so each ran its own sweep)
    assert res[(False, "BSP")][2] != res[(False, "SP")][2] or rel(res[(False, "BSP")][0][:2], res[(False, "SP")][0][:2]) > 1e-12
    p.close()


@pytest.mark.parametrize("mode", ["barrier", "dependency"])
@pytest.mark.parametrize("sched", ["BSP", "SP", "BSP_NONOVERLAP"])
def test_persistent_sweep_gives_the_same_solve(H, sched, mode):
    """persistent: the interface stages of each sweep in one cooperative launch, with grid
    barriers between stages or with per-item dependencies; the same items with the same
    arithmetic, so the same iterates (the dependency-driven form also inside the
    device-driven loop)."""
    w = CASES["uneven_4x3"]()
    p, _ = make(H, w, "c64")
    f = cuda(W.random_complex((2, w.N), 24))
    kw = dict(tol=1e-9, restart=30, maxit=200, sched=sched, inner_maxit=60, inner_tol=1e-3)
    u0, i0, _ = p.solve(f, **kw)
    u1, i1, _ = p.solve(f, persistent=mode, **kw)
    print(f"{sched} {mode}: its {[i[0] for i in i0]} vs {[i[0] for i in i1]}, rel {rel(u1.cpu().numpy(), u0.cpu().numpy()):.1e}")
    assert [i[0] for i in i0] == [i[0] for i in i1]
    assert rel(u1.cpu().numpy(), u0.cpu().numpy()) <= 1e-9
    p.close()


def test_interface_krylov_without_boundary_operators(H):
    """The interface operator S and the sweep by full local solves (no K)."""
    w = CASES["tiny_2x2"]()
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), w.N1, w.N2, w.xcuts, w.ycuts,
                  boundary_operators=False).factor("c64")
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    u, info, _ = p.solve(cuda(w.f), tol=1e-9, restart=30, maxit=100, inner_maxit=40, inner_tol=1e-4)
    ref = spla.spsolve(A, w.h ** 2 * w.f[0])
    assert info[0][1] <= 1e-9 and rel(u.cpu().numpy()[0], ref) <= 1e-5
    p.close()


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_graph_replay_gives_the_same_solve(H, prec):
    """use_graph: the preconditioner replayed from captured CUDA graphs runs the same
    kernels on the same data, so the iteration counts and residuals are identical."""
    w = CASES["uneven_4x3"]()
    p, _ = make(H, w, prec)
    f = cuda(W.random_complex((2, w.N), 21))
    u0, i0, _ = p.solve(f, tol=1e-9, restart=30, maxit=400)
    n0 = H.launch_count()
    u1, i1, _ = p.solve(f, tol=1e-9, restart=30, maxit=400, use_graph=True)
    n1 = H.launch_count()
    u2, i2, _ = p.solve(f, tol=1e-9, restart=30, maxit=400, use_graph=True)      # replays cached graphs
    assert i0 == i1 == i2
    assert rel(u1.cpu().numpy(), u0.cpu().numpy()) <= 1e-12
    assert rel(u2.cpu().numpy(), u0.cpu().numpy()) <= 1e-12
    assert H.launch_count() - n1 == n1 - n0          # replays count the kernels they run
    p.close()


def test_misfit_gradient_matches_direct_adjoint(H):
    n = 63
    w = W.workload("custom", n=n, N1=2, N2=2, medium="layered", seed=3, nrhs=3)
    rec = np.arange((n - 1) * n + 1, n * n, 4)
    rng = np.random.default_rng(1)
    d = (rng.normal(size=(3, len(rec))) + 1j * rng.normal(size=(3, len(rec)))) * 1e-4
    J, g, U = misfit_gradient_direct(w.n, w.h, w.omega, w.m2, w.f, rec, d)
    for prec, tol in (("c128", 1e-7), ("c64", 1e-7)):
        p, _ = make(H, w, prec)
        Jg, gg, ug = p.misfit_grad(cuda(w.f), torch.as_tensor(rec), cuda(d), tol=1e-11, maxit=2000)
        gg = gg.cpu().numpy()
        print(f"misfit {prec}: J rel {abs(Jg - J) / J:.2e}, grad rel {rel(gg, g):.2e}")
        assert abs(Jg - J) <= tol * J
        assert rel(gg, g) <= 1e-6
        p.close()


def test_autograd_function_backward_is_the_adjoint_gradient(H):
    n = 47
    w = W.workload("custom", n=n, N1=2, N2=2, medium="layered", seed=9, nrhs=2)
    rec = np.arange((n - 1) * n, n * n, 3)
    d = np.zeros((2, len(rec)), dtype=complex)
    J, g, _ = misfit_gradient_direct(w.n, w.h, w.omega, w.m2, w.f, rec, d)
    m2 = cuda(w.m2, torch.float64).requires_grad_(True)
    spec = dict(n=n, h=w.h, omega=w.omega, N1=2, N2=2, xcuts=w.xcuts, ycuts=w.ycuts, prec="c128", tol=1e-11)
    Jt = H.MisfitFn.apply(m2, cuda(w.f), torch.as_tensor(rec), cuda(d), spec)
    (2.0 * Jt).backward()
    assert abs(Jt.item() - J) <= 1e-7 * J
    assert rel(m2.grad.cpu().numpy(), 2.0 * g) <= 1e-6


def test_state_and_argument_errors(H):
    w = CASES["tiny_2x2"]()
    p = H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), 2, 2, w.xcuts, w.ycuts)
    with pytest.raises(H.HelmError) as e:
        p.precond_apply(cuda(np.zeros(w.N)))
    assert e.value.status == 4
    with pytest.raises(H.HelmError) as e:
        p.solve(cuda(w.f))
    assert e.value.status == 4
    p.factor("c64")
    with pytest.raises(H.HelmError) as e:
        p.solve(cuda(w.f), restart=0)
    assert e.value.status == 1
    u, info, _ = p.solve(cuda(w.f), maxit=2, raise_on_noconv=False)
    assert info[0][0] == 2 and info[0][1] > 1e-6
    with pytest.raises(H.HelmError) as e:
        p.solve(cuda(w.f), maxit=2)
    assert e.value.status == 5
    with pytest.raises(H.HelmError):
        H.Problem(w.n, w.n, w.h, w.omega, cuda(w.m2, torch.float64), 2, 2, [0, 70, 60], [0, 64, 127])
    p.close()
