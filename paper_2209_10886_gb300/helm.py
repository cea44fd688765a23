"""ctypes binding of libhelm (include/helm.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch
tensors to device pointers, passes the current CUDA stream and turns status
codes into exceptions.  There is no CPU fallback: if the shared library is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import re

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# HELM_LIBRARY=check loads the bounds-checking build (build.build(variant="check"))
LIB_PATH = os.path.join(_HERE, "libhelm_check.so" if os.environ.get("HELM_LIBRARY") == "check" else "libhelm.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "helm.h")

PREC = {"c128": 0, "c64": 1}
SCHED = {"BSP": 0, "SP": 1, "BSP_NONOVERLAP": 2}
TRANSMISSION = {"optimized": 0, "impedance": 1, "habc": 2}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_STATE", 5: "ERR_NO_CONVERGENCE",
          6: "ERR_TIMEOUT", 7: "ERR_UNSUPPORTED"}


class HelmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class HelmOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("maxit", ctypes.c_int), ("tol", ctypes.c_double),
                ("x0_given", ctypes.c_int), ("sched", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("hist", ctypes.POINTER(ctypes.c_double)), ("ortho", ctypes.c_int),
                ("inner_maxit", ctypes.c_int), ("inner_restart", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("persistent", ctypes.c_int), ("inner_hist", ctypes.POINTER(ctypes.c_double)),
                ("inner_fp64", ctypes.c_int), ("wait_cycles", ctypes.c_longlong)]


class HelmSetupOpts(ctypes.Structure):
    _fields_ = [("transmission", ctypes.c_int), ("tc_scale", ctypes.c_double),
                ("boundary_operators", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("tc_min_rhs", ctypes.c_int), ("autotune", ctypes.c_int), ("tc_iface_min_ctas", ctypes.c_int),
                ("device_budget", ctypes.c_size_t), ("n_pade", ctypes.c_int), ("pade_phi", ctypes.c_double),
                ("tc_factor", ctypes.c_int), ("sym_k", ctypes.c_int)]


class HelmInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("relres", ctypes.c_double)]


_lib = None
_vp, _i, _d, _ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong


def lib():
    """Load libhelm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2209_10886_gb300.build.build()"
                           + (' (variant="check")' if LIB_PATH.endswith("_check.so") else ""))
    L = ctypes.CDLL(LIB_PATH)
    L.helm_default_opts.argtypes = [ctypes.POINTER(HelmOpts)]
    L.helm_default_opts.restype = None
    L.helm_default_setup_opts.argtypes = [ctypes.POINTER(HelmSetupOpts)]
    L.helm_default_setup_opts.restype = None
    L.helm_setup.argtypes = [_i, _i, _d, _d, _vp, _i, _i, _vp, _vp, ctypes.POINTER(HelmSetupOpts),
                             ctypes.POINTER(_vp)]
    L.precond_factor.argtypes = [_vp, _i, _vp]
    L.precond_apply.argtypes = [_vp, _i, _vp, _vp, _i, _vp]
    L.helm_matvec.argtypes = [_vp, _vp, _vp, _i, _vp]
    L.gmres_solve.argtypes = [_vp, _vp, _vp, _i, ctypes.POINTER(HelmOpts), ctypes.POINTER(HelmInfo), _vp]
    L.misfit_grad.argtypes = [_vp, _vp, _i, _vp, _i, _vp, ctypes.POINTER(HelmOpts), ctypes.POINTER(_d), _vp, _vp, _vp]
    L.helm_destroy.argtypes = [_vp]
    L.helm_last_error.argtypes = []
    L.helm_last_error.restype = ctypes.c_char_p
    L.helm_schedule_info.argtypes = [_i, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]
    L.helm_problem_info.argtypes = [_vp, ctypes.POINTER(_ll), ctypes.POINTER(_i), ctypes.POINTER(_ll),
                                    ctypes.POINTER(_ll)]
    for name in ("helm_setup", "precond_factor", "precond_apply", "helm_matvec", "gmres_solve", "misfit_grad",
                 "helm_destroy", "helm_schedule_info", "helm_problem_info"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def header_functions():
    """Names of the functions declared in include/helm.h."""
    txt = open(HEADER_PATH).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    txt = re.sub(r"^\s*#.*$", "", txt, flags=re.M)          # preprocessor lines
    return sorted(set(re.findall(r"\b(\w+)\s*\([^;{]*\)\s*;", txt)) - {"if", "while", "for", "sizeof"})


def _check(status, what=""):
    if status != 0:
        raise HelmError(status, lib().helm_last_error().decode() or what)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _as_fields(x: torch.Tensor, N: int, name: str) -> torch.Tensor:
    if not x.is_cuda or x.dtype != torch.complex128:
        raise TypeError(f"{name} must be a complex128 CUDA tensor")
    if x.numel() % N != 0:
        raise ValueError(f"{name} must hold a multiple of N = {N} values")
    return x.contiguous()


def schedule_info(N1: int, N2: int, sched: str = "BSP"):
    """(sweep steps, stage launches) per preconditioner application (host only)."""
    steps, stages = _i(), _i()
    _check(lib().helm_schedule_info(N1, N2, SCHED[sched], ctypes.byref(steps), ctypes.byref(stages)))
    return steps.value, stages.value


def default_opts(**kw) -> HelmOpts:
    o = HelmOpts()
    lib().helm_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "sched":
            v = SCHED[v] if isinstance(v, str) else v
        setattr(o, k, v)
    return o


class Problem:
    """A discretised Helmholtz problem with its checkerboard decomposition.

    ``m2``: squared slowness (float64, n_x*n_y values, CUDA).  ``xcuts`` /
    ``ycuts``: node offsets of the subdomain columns / rows (length N1+1 /
    N2+1) or None for an even split.  The remaining keywords are the fields of
    ``helm_setup_opts``: ``transmission`` ("optimized" or "impedance") and
    ``tc_scale``; ``boundary_operators``; ``tensor_cores`` (True / "3xtf32",
    "tf32", False) with ``tc_min_rhs``; ``autotune`` (time the interface-stage
    shapes at the first application per RHS count); ``tc_iface_min_ctas``
    (interface stages of fewer CTAs keep the CUDA-core form when the tensor-core
    form is chosen; -1: two per SM); ``device_budget`` (bytes the handle's large arrays
    may take, 0: no limit); ``n_pade`` and ``pade_phi`` of the "habc" transmission (the
    Pade HABC of the paper's experiments, with ``tc_scale`` the Robin parameter of the
    factored base problem); ``tc_factor`` (complex64 factorisation with tensor-core
    trailing updates, subdomains at most 128 nodes wide); ``sym_k`` (complex64 interface
    stages of one RHS that apply every subdomain's whole K stream the packed symmetric
    operators).
    """

    def __init__(self, n_x, n_y, h, omega, m2, N1, N2, xcuts=None, ycuts=None,
                 transmission="optimized", tc_scale=1.0, boundary_operators=True, tensor_cores=True,
                 tc_min_rhs=16, autotune=True, tc_iface_min_ctas=-1, device_budget=0, n_pade=8,
                 pade_phi=math.pi / 3, tc_factor=True, sym_k=True):
        L = lib()
        if not (m2.is_cuda and m2.dtype == torch.float64 and m2.numel() == n_x * n_y):
            raise TypeError("m2 must be a float64 CUDA tensor with n_x*n_y values")
        m2 = m2.contiguous()
        tcm = {False: 0, True: 1, "3xtf32": 1, "tf32": 2}[tensor_cores]
        so = HelmSetupOpts(TRANSMISSION[transmission], float(tc_scale), int(bool(boundary_operators)), tcm,
                           int(tc_min_rhs), int(bool(autotune)), int(tc_iface_min_ctas), int(device_budget),
                           int(n_pade), float(pade_phi), int(bool(tc_factor)), int(bool(sym_k)))
        xc = (ctypes.c_int * (N1 + 1))(*[int(v) for v in xcuts]) if xcuts is not None else None
        yc = (ctypes.c_int * (N2 + 1))(*[int(v) for v in ycuts]) if ycuts is not None else None
        h_ = ctypes.c_void_p()
        torch.cuda.current_stream().synchronize()
        _check(L.helm_setup(n_x, n_y, float(h), float(omega), _ptr(m2), N1, N2, xc, yc, ctypes.byref(so),
                            ctypes.byref(h_)))
        self._h = h_
        self.n_x, self.n_y, self.h, self.omega, self.N1, self.N2 = n_x, n_y, h, omega, N1, N2
        self.N = n_x * n_y
        self.m2 = m2

    # ----------------------------------------------------------------- info
    def factor_on_tensor_cores(self) -> bool:
        """True when the last factorisation ran its trailing updates on the tensor cores."""
        L = lib()
        L.helm_factor_on_tensor_cores.restype = ctypes.c_int
        L.helm_factor_on_tensor_cores.argtypes = [_vp]
        return bool(L.helm_factor_on_tensor_cores(self._h))

    def iface_symmetric(self, nrhs=1) -> bool:
        """True when interface stages with nrhs RHS apply the packed symmetric operators."""
        L = lib()
        L.helm_iface_symmetric.restype = ctypes.c_int
        L.helm_iface_symmetric.argtypes = [_vp, ctypes.c_int]
        return bool(L.helm_iface_symmetric(self._h, int(nrhs)))

    def info(self):
        n, ns, nt, fb = _ll(), _i(), _ll(), _ll()
        _check(lib().helm_problem_info(self._h, ctypes.byref(n), ctypes.byref(ns), ctypes.byref(nt),
                                       ctypes.byref(fb)))
        return dict(n_unknowns=n.value, n_subdomains=ns.value, n_trace=nt.value, factor_bytes=fb.value)

    # -------------------------------------------------------------- compute
    def factor(self, prec="c64", stream=None):
        _check(lib().precond_factor(self._h, PREC[prec], _stream(stream)))
        self.prec = prec
        return self

    def precond_apply(self, r, z=None, sched="BSP", stream=None):
        r = _as_fields(r, self.N, "r")
        z = torch.empty_like(r) if z is None else z
        _check(lib().precond_apply(self._h, SCHED[sched], _ptr(r), _ptr(z), r.numel() // self.N, _stream(stream)))
        return z

    def matvec(self, u, Au=None, stream=None):
        u = _as_fields(u, self.N, "u")
        Au = torch.empty_like(u) if Au is None else Au
        _check(lib().helm_matvec(self._h, _ptr(u), _ptr(Au), u.numel() // self.N, _stream(stream)))
        return Au

    def solve(self, f, u=None, restart=50, maxit=1000, tol=1e-6, sched="BSP", x0=None, history=False,
              stream=None, raise_on_noconv=True, use_graph=False, inner_maxit=0, inner_restart=100, inner_tol=1e-4,
              persistent=False, ortho="mgs", inner_fp64=False, inner_history=False, wait_cycles=0):
        """Solve A u = h^2 f (FP64 FGMRES); returns (u, [(iters, relres)], history or None).
        ortho: "mgs" (volume default), "cgs2" or "cgs2_split" (see helm.h); inner_fp64: FP64
        interface Krylov vectors with complex64 factors (default: complex64 vectors);
        inner_history: keep the interface residual history of the first preconditioner
        application in self.last_inner_history (one list per RHS); persistent: False (stage
        launches), True / "barrier" or "dependency" (one cooperative launch per sweep, see
        helm.h); wait_cycles: grid-barrier limit of the Gram-Schmidt kernels (0: ~1 s)."""
        f = _as_fields(f, self.N, "f")
        nrhs = f.numel() // self.N
        u = torch.empty_like(f) if u is None else u
        if x0 is not None:
            u.copy_(x0)
        hist = (ctypes.c_double * (maxit * nrhs))() if history else None
        o = default_opts(restart=restart, maxit=maxit, tol=tol, sched=sched, x0_given=int(x0 is not None),
                         use_graph=int(bool(use_graph)), inner_maxit=int(inner_maxit),
                         inner_restart=int(inner_restart), inner_tol=float(inner_tol),
                         persistent={False: 0, True: 1, "barrier": 1, "dependency": 2}.get(persistent, persistent),
                         ortho=ORTHO[ortho], inner_fp64=int(bool(inner_fp64)), wait_cycles=int(wait_cycles))
        if hist is not None:
            o.hist = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
        ihist = (ctypes.c_double * (max(1, int(inner_maxit)) * nrhs))() if inner_history else None
        if ihist is not None:
            o.inner_hist = ctypes.cast(ihist, ctypes.POINTER(ctypes.c_double))
        info = (HelmInfo * nrhs)()
        st = lib().gmres_solve(self._h, _ptr(f), _ptr(u), nrhs, ctypes.byref(o), info, _stream(stream))
        if st != 0 and (raise_on_noconv or st != 5):
            _check(st)
        out = [(info[k].iters, info[k].relres) for k in range(nrhs)]
        if ihist is not None:
            m = max(1, int(inner_maxit))
            rows = [list(ihist[k * m:(k + 1) * m]) for k in range(nrhs)]
            # steps not taken keep the buffer's zeros
            self.last_inner_history = [r[:max([i + 1 for i, v in enumerate(r) if v != 0.0] or [0])] for r in rows]
        hh = None
        if hist is not None:
            hh = [[hist[k * maxit + j] for j in range(out[k][0])] for k in range(nrhs)]
        return u, out, hh

    def misfit_grad(self, f, rec_idx, d, restart=50, maxit=1000, tol=1e-6, sched="BSP", stream=None):
        """(J, grad_m2, u) of J = 1/2 sum_s ||P u_s - d_s||^2 by the adjoint-state method."""
        f = _as_fields(f, self.N, "f")
        nsrc = f.numel() // self.N
        rec = rec_idx.to(device=f.device, dtype=torch.int32).contiguous()
        d = d.to(device=f.device, dtype=torch.complex128).contiguous()
        if d.numel() != nsrc * rec.numel():
            raise ValueError("d must hold nsrc*nrec values")
        grad = torch.empty(self.N, dtype=torch.float64, device=f.device)
        u = torch.empty_like(f)
        J = ctypes.c_double()
        o = default_opts(restart=restart, maxit=maxit, tol=tol, sched=sched)
        _check(lib().misfit_grad(self._h, _ptr(f), nsrc, _ptr(rec), rec.numel(), _ptr(d), ctypes.byref(o),
                                 ctypes.byref(J), _ptr(grad), _ptr(u), _stream(stream)))
        return J.value, grad, u

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().helm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MisfitFn(torch.autograd.Function):
    """``J = MisfitFn.apply(m2, f, rec_idx, d, spec)``: the misfit of the sources
    ``f`` at the receivers ``rec_idx`` for the squared slowness ``m2``; its
    backward returns ``grad_output * dJ/dm2`` computed by the adjoint kernels.

    ``spec``: dict with n, h, omega, N1, N2, xcuts, ycuts and optional prec,
    restart, tol, sched, transmission.
    """

    @staticmethod
    def forward(ctx, m2, f, rec_idx, d, spec):
        n = spec["n"]
        p = Problem(n, n, spec["h"], spec["omega"], m2.detach(), spec["N1"], spec["N2"], spec.get("xcuts"),
                    spec.get("ycuts"), transmission=spec.get("transmission", "optimized"))
        try:
            p.factor(spec.get("prec", "c64"))
            J, grad, _ = p.misfit_grad(f, rec_idx, d, restart=spec.get("restart", 50), tol=spec.get("tol", 1e-6),
                                       maxit=spec.get("maxit", 2000), sched=spec.get("sched", "BSP"))
        finally:
            p.close()
        ctx.save_for_backward(grad)
        return torch.tensor(J, dtype=torch.float64, device=m2.device)

    @staticmethod
    def backward(ctx, grad_output):
        (grad,) = ctx.saved_tensors
        return grad_output * grad, None, None, None, None


def habc_side_operator(kappa, h: float, n_pade: int = 8, phi: float = math.pi / 3):
    """The HABC transmission operator of one interface side as an L x L complex128
    array (host only; see ``helm_habc_side_operator`` in include/helm.h)."""
    k = np.ascontiguousarray(kappa, dtype=np.float64).reshape(-1)
    L = k.size
    T = np.empty((L, L), dtype=np.complex128)
    fn = lib().helm_habc_side_operator
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
    _check(fn(k.ctypes.data, L, float(h), int(n_pade), float(phi), T.ctypes.data))
    return T


# ------------------------------------------------- sources over several ranks
def source_shard(nsrc: int, rank: int, world: int) -> range:
    """The sources of ``rank`` when ``nsrc`` sources are dealt to ``world`` ranks in
    contiguous blocks (the first ``nsrc % world`` ranks take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    q, r = divmod(int(nsrc), int(world))
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


def reduce_misfit(J: float, grad: "torch.Tensor", group=None):
    """Sum a rank's misfit and gradient over the ranks of ``group`` (the default
    process group when None; unchanged without torch.distributed): the misfit and
    its gradient are sums over the sources, so source-parallel inversion needs this
    one all-reduce of N + 1 doubles and nothing else."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return J, grad
    buf = torch.cat([grad.reshape(-1).to(torch.float64),
                     torch.tensor([J], dtype=torch.float64, device=grad.device)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return float(buf[-1]), buf[:-1].reshape(grad.shape)


def misfit_grad_sharded(problem: "Problem", f, rec_idx, d, group=None, **kw):
    """``(J, grad_m2, u)`` over the sources of all ranks: each rank passes its own
    sources (``f``: its rows, ``d``: their data; see :func:`source_shard`) and gets
    the total misfit and gradient; ``u`` stays the rank's own fields."""
    J, grad, u = problem.misfit_grad(f, rec_idx, d, **kw)
    J, grad = reduce_misfit(J, grad, group)
    return J, grad, u


# ------------------------------------------------------------------ profiling
class HelmKStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


ORTHO = {"mgs": 0, "cgs2": 1, "cgs2_split": 2}
KERNEL_CLASS = {"stage": 0, "matvec": 1, "ortho": 2, "other": 3, "trace": 4}


def launch_count() -> int:
    """CUDA kernel launches issued by the library in this process."""
    L = lib()
    L.helm_launch_count.restype = ctypes.c_longlong
    return int(L.helm_launch_count())


def inner_steps(problem: "Problem") -> int:
    """Interface Krylov steps taken inside the preconditioner applications of a problem."""
    L = lib()
    L.helm_inner_steps.restype = ctypes.c_longlong
    L.helm_inner_steps.argtypes = [_vp]
    return int(L.helm_inner_steps(problem._h))


def iface_shape(problem: "Problem", nrhs: int) -> dict:
    """Launch shape of the interface-stage kernel for nrhs RHS (autotuned or the fixed rules)."""
    L = lib()
    L.helm_iface_shape.restype = ctypes.c_int
    L.helm_iface_shape.argtypes = [_vp, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 6
    v = [ctypes.c_int() for _ in range(6)]
    _check(L.helm_iface_shape(problem._h, int(nrhs), *[ctypes.byref(x) for x in v]))
    return {"rhs_per_block": v[0].value, "staged": v[1].value, "ctas_per_sm": v[2].value,
            "tensor_cores": v[3].value, "tensor_rhs_per_cta": v[4].value, "tuned": bool(v[5].value)}


def stage_shape(problem: "Problem", nrhs: int) -> dict:
    """Launch shape of the full-stage kernels for nrhs RHS (autotuned, or 0s for the rules)."""
    L = lib()
    L.helm_stage_shape.restype = ctypes.c_int
    L.helm_stage_shape.argtypes = [_vp, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 4
    v = [ctypes.c_int() for _ in range(4)]
    _check(L.helm_stage_shape(problem._h, int(nrhs), *[ctypes.byref(x) for x in v]))
    return {"ctas_per_subdomain": v[0].value, "chunk_kb": v[1].value, "tensor_rhs_per_cta": v[2].value,
            "tuned": bool(v[3].value)}


def check_bounds_report(reset: bool = False) -> dict:
    """Failed bounds checks of the bounds-checking build (HELM_LIBRARY=check) since the last
    reset: their count and the first one; checking_build is False for the normal build."""
    L = lib()
    L.helm_check_bounds_report.restype = ctypes.c_int
    L.helm_check_bounds_report.argtypes = [ctypes.POINTER(_ll), ctypes.POINTER(ctypes.c_ulonglong),
                                           ctypes.POINTER(_ll), ctypes.POINTER(_i), ctypes.c_char_p, _i, _i]
    v, b, ln = _ll(), _ll(), _i()
    a = ctypes.c_ulonglong()
    unit = ctypes.create_string_buffer(256)
    rc = L.helm_check_bounds_report(ctypes.byref(v), ctypes.byref(a), ctypes.byref(b), ctypes.byref(ln), unit, 256,
                                    int(bool(reset)))
    if rc < 0:
        raise HelmError(2, "helm_check_bounds_report: CUDA error")
    return {"checking_build": rc == 1, "violations": v.value, "first_addr": a.value, "first_bytes": b.value,
            "first_line": ln.value, "unit": unit.value.decode()}


def check_bounds_selftest():
    """The checking build's check on a 256-byte allocation: (whole allocation passes, the
    byte past its end passes, a range straddling its end passes); None for the normal build."""
    L = lib()
    L.helm_check_bounds_selftest.restype = ctypes.c_int
    L.helm_check_bounds_selftest.argtypes = [ctypes.POINTER(_i)]
    res = (_i * 3)()
    rc = L.helm_check_bounds_selftest(res)
    if rc < 0:
        raise HelmError(2, "helm_check_bounds_selftest: CUDA error")
    return tuple(bool(x) for x in res) if rc == 1 else None


def profile(problem: "Problem", on: bool = True):
    _check(lib().helm_profile(problem._h, int(on)))


def profile_read(problem: "Problem", kind: str):
    """(launches, summed event ms, algorithmic bytes, algorithmic flops) of one kernel class."""
    L = lib()
    L.helm_profile_read.argtypes = [_vp, _i, ctypes.POINTER(HelmKStat)]
    st = HelmKStat()
    _check(L.helm_profile_read(problem._h, KERNEL_CLASS[kind], ctypes.byref(st)))
    return st.launches, st.ms, st.bytes, st.flops
