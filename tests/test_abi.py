"""CPU checks of the C ABI: the library loads, exports every function the
header declares, and its host-side scheduler reproduces the paper's step
counts.  No compute call needs a GPU here."""
import ctypes
import os

import numpy as np
import pytest

from paper_2209_10886_gb300 import build as B


@pytest.fixture(scope="module")
def L():
    B.build()
    from paper_2209_10886_gb300 import helm
    return helm.lib()


def test_library_exports_every_declared_function(L):
    from paper_2209_10886_gb300 import helm
    names = helm.header_functions()
    assert {"helm_setup", "precond_factor", "precond_apply", "gmres_solve", "misfit_grad", "helm_matvec",
            "helm_destroy", "helm_last_error"} <= set(names)
    for n in names:
        assert hasattr(L, n), n


def test_scheduler_reproduces_table1(L, golden_dir):
    from paper_2209_10886_gb300 import schedule_info
    rows = np.loadtxt(os.path.join(golden_dir, "table1_steps.txt"), dtype=int, ndmin=2)
    for N1, N2, sp_ns, bsp_ns in rows:
        assert schedule_info(N1, N2, "SP")[0] == sp_ns
        assert schedule_info(N1, N2, "BSP")[0] == bsp_ns


@pytest.mark.parametrize("N1,N2", [(1, 1), (2, 2), (8, 8), (12, 12), (16, 16), (5, 10), (3, 7), (7, 3), (1, 5)])
def test_scheduler_matches_oracle_schedule(L, N1, N2):
    """Step counts of the C++ scheduler equal the oracle's (Sections 4-5; BSP also with
    non-overlapping bands), and the stage count is steps + lifting + reconstruction
    (+ residual for BSP)."""
    from oracle import schedule_steps
    from paper_2209_10886_gb300 import schedule_info
    for kind in ("SP", "BSP", "BSP_NONOVERLAP"):
        steps, stages = schedule_info(N1, N2, kind)
        if N1 * N2 == 1:
            assert (steps, stages) == (0, 1)
            continue
        if kind == "BSP_NONOVERLAP":
            assert steps == schedule_steps(N1, N2, "BSP", overlap=False) == 2 * (N1 - 1)
        else:
            assert steps == schedule_steps(N1, N2, kind)
        assert stages == steps + 2 + (kind != "SP")


def test_invalid_arguments_are_rejected_without_gpu(L):
    from paper_2209_10886_gb300 import helm
    s = ctypes.c_int()
    assert L.helm_schedule_info(0, 3, 0, ctypes.byref(s), None) == 1
    assert b"N1" in L.helm_last_error()
    assert L.helm_setup(0, 5, 0.1, 1.0, None, 1, 1, None, None, None, ctypes.byref(ctypes.c_void_p())) == 1
    assert L.helm_destroy(None) == 0


def _header_struct_fields(name):
    """Field names of the typedef struct `name` in include/helm.h, in order."""
    import re
    from paper_2209_10886_gb300 import helm
    txt = re.sub(r"/\*.*?\*/", "", open(helm.HEADER_PATH).read(), flags=re.S)
    body = re.search(r"typedef\s+struct\s*\{([^}]*)\}\s*" + name + r"\s*;", txt).group(1)
    fields = []
    for decl in filter(None, (d.strip() for d in body.split(";"))):
        # "int a, b" / "double* hist" / "int x[4]": the identifier ending each declarator
        fields += [re.findall(r"(\w+)\s*$", part.split("[")[0])[0] for part in decl.split(",")]
    return fields


@pytest.mark.parametrize("cname,pyname", [("helm_setup_opts", "HelmSetupOpts"), ("helm_opts", "HelmOpts")])
def test_binding_structs_follow_the_header(L, cname, pyname):
    """The ctypes structures the binding passes across the ABI have the header's fields
    in the header's order."""
    from paper_2209_10886_gb300 import helm
    py = [f[0] for f in getattr(helm, pyname)._fields_]
    assert py == _header_struct_fields(cname)


def test_shape_query_rejects_a_null_handle_without_gpu(L):
    """helm_iface_shape through the binding (all eight arguments) reports HELM_ERR_ARG
    for a NULL handle."""
    from paper_2209_10886_gb300 import helm

    class NoProblem:
        _h = None
    with pytest.raises(helm.HelmError) as e:
        helm.iface_shape(NoProblem(), 4)
    assert e.value.status == 1 and "NULL" in str(e.value)


def test_habc_side_operator_matches_the_oracle_without_gpu(L):
    """The library's host builder of the HABC side operator (C++, its own LU) equals
    the oracle's NumPy one; N = 0 without rotation is i diag(kappa); bad arguments
    give HELM_ERR_ARG."""
    from oracle import habc
    from paper_2209_10886_gb300 import helm
    rng = np.random.default_rng(3)
    for Lside, N, phi in ((37, 8, np.pi / 3), (5, 3, 0.4), (1, 8, np.pi / 3), (128, 8, np.pi / 3)):
        kappa = 40.0 + 10.0 * rng.random(Lside)
        T = helm.habc_side_operator(kappa, 0.01, N, phi)
        ref = habc.side_operator(kappa, 0.01, N, phi)
        assert np.linalg.norm(T - ref) <= 1e-12 * np.linalg.norm(ref), (Lside, N)
    kappa = 30.0 + rng.random(9)
    assert np.allclose(helm.habc_side_operator(kappa, 0.02, 0, 0.0), np.diag(1j * kappa), rtol=0, atol=1e-14)
    with pytest.raises(helm.HelmError):
        helm.habc_side_operator(np.array([1.0, -2.0]), 0.01)
    with pytest.raises(helm.HelmError):
        helm.habc_side_operator(np.array([1.0, 2.0]), 0.0)


def test_normal_build_reports_no_bounds_checking_without_gpu(L):
    """The diagnostics of the bounds-checking build exist in the normal build too, where
    they report that no check is compiled in and touch no device."""
    from paper_2209_10886_gb300 import helm
    if os.environ.get("HELM_LIBRARY") == "check":
        pytest.skip("the checking build is loaded")
    r = helm.check_bounds_report()
    assert r["checking_build"] is False and r["violations"] == 0
    assert helm.check_bounds_selftest() is None


def test_packed_operator_query_rejects_a_null_handle_without_gpu(L):
    L.helm_iface_symmetric.restype = ctypes.c_int
    L.helm_iface_symmetric.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert L.helm_iface_symmetric(None, 1) == 0
