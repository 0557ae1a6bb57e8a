"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/diagmg.h declares, rejects invalid descriptions before
touching CUDA, and the binding has no CPU fallback."""

import ctypes
import os

import pytest

from paper_math_9907190_gb300 import _native as N
from paper_math_9907190_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.lib()


def test_library_exports_every_declared_function(lib):
    declared = N.header_functions()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    assert set(N.SIGNATURES) <= set(declared)


def _desc(**kw):
    d = N.mg_desc()
    base = dict(dim=2, n=63, pitch=65, hierarchy=N.MG_DIAG, order=2, precision=N.MG_FP64, coarsest=3)
    base.update(kw)
    for k, v in base.items():
        setattr(d, k, v)
    for i in range(4):
        d.omega[i] = 1.0
    return d


@pytest.mark.parametrize("bad", [
    dict(dim=1), dict(dim=4), dict(n=64), dict(n=1), dict(n=0), dict(n=-1), dict(pitch=64),
    dict(hierarchy=2), dict(order=3), dict(precision=7), dict(coarsest=2), dict(coarsest=127),
    dict(dim=3, n=15, pitch=17, coarsest=15), dict(coarsest=15), dict(dim=3, n=31, pitch=33, coarsest=5),
])
def test_create_rejects_invalid_descriptions(lib, bad):
    h = ctypes.c_void_p()
    st = lib.mg_create(ctypes.byref(h), ctypes.byref(_desc(**bad)))
    assert st == N.MG_EINVAL and not h.value


def test_nan_omega_rejected(lib):
    d = _desc()
    d.omega[1] = float("nan")
    h = ctypes.c_void_p()
    assert lib.mg_create(ctypes.byref(h), ctypes.byref(d)) == N.MG_EINVAL


def test_null_arguments_rejected(lib):
    assert lib.mg_create(None, ctypes.byref(_desc())) == N.MG_EINVAL
    assert lib.mg_num_levels(None, None) == N.MG_EINVAL
    assert lib.mg_level_info(None, 0, None, None) == N.MG_EINVAL
    assert lib.mg_residual(None, None, None, 1.0, 2, None, None, None) == N.MG_EINVAL
    assert lib.mg_restrict_diag(None, 0, None) == N.MG_EINVAL
    assert lib.mg_jacobi_prolong(None, 0, None, None) == N.MG_EINVAL
    assert lib.mg_coarse_solve(None, None) == N.MG_EINVAL
    assert lib.mg_vcycle(None, None, None, None) == N.MG_EINVAL
    assert lib.mg_solve(None, None, None, 1e-10, 10, None, None, None, None) == N.MG_EINVAL
    assert lib.mg_solve_zero(None, None, None, 1e-10, 10, None, None, None, None) == N.MG_EINVAL
    assert lib.mg_level_get(None, 0, 0, None, None) == N.MG_EINVAL
    assert lib.mg_solve_host(None, None, None, None, 1e-10, 10, None, None, None) == N.MG_EINVAL
    assert lib.mg_solve_host_many(None, 2, None, None, 1e-10, 10, None, None, None) == N.MG_EINVAL
    assert lib.mg_fp64_rate(None, None, None) == N.MG_EINVAL
    assert lib.mg_batch_status(None, None) == N.MG_EINVAL
    assert lib.mg_set_gamma(None, 2) == N.MG_EINVAL
    assert lib.mg_destroy(None) == N.MG_OK


def test_noalloc_rejects_misaligned_grids_before_touching_cuda(lib):
    """Grid pointers must sit on FP64 element boundaries; the check comes
    before any CUDA call, so it runs without a GPU (the addresses are never
    dereferenced)."""
    f = ctypes.c_void_p(0x10000)
    for bad in (0x10001, 0x10004, 0x1000C):
        p = ctypes.c_void_p(bad)
        h = 1.0 / 64
        assert lib.mg_residual_noalloc(2, 63, 65, ctypes.c_double(h), 2, p, f, None, None, None) == N.MG_EINVAL
        assert lib.mg_residual_noalloc(2, 63, 65, ctypes.c_double(h), 2, f, p, None, None, None) == N.MG_EINVAL
        assert lib.mg_residual_noalloc(2, 63, 65, ctypes.c_double(h), 2, f, f, p, None, None) == N.MG_EINVAL


def test_strerror(lib):
    for st in (0, -1, -2, -3, -4, -5, -6):
        assert lib.mg_strerror(st)
    assert lib.mg_strerror(N.MG_ENOCONV) == b"not converged within max_cycles"


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(N, "_lib", None)
    monkeypatch.setattr(N, "LIB_PATH", os.path.join(os.path.dirname(N.LIB_PATH), "missing-libdiagmg.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        N.lib()


def _kernel_heads(path):
    """(name, statements before the first wait) of every __global__ function."""
    import re
    src = open(path).read()
    out = []
    for m in re.finditer(r"__global__[^{;]*?\b(k_\w+)\s*\(", src):
        body = src.index("{", m.end())
        head = []
        for line in src[body + 1:].split("\n"):
            t = line.strip()
            if "pdl_wait()" in t or "stop(" in t:
                break
            t = t.split("//")[0].strip()
            if t:
                head.append(t)
            if len(head) > 40:
                break
        out.append((m.group(1), head))
    return out


def test_every_context_kernel_waits_before_touching_memory():
    """With programmatic dependent launch a kernel starts while the previous
    one finishes, so each kernel a context launches must wait (pdl_wait, or
    stop, which calls it) before it reads or writes global memory: only
    declarations, shared arrays and index arithmetic may come first."""
    import re
    csrc = os.path.join(os.path.dirname(N.__file__), "csrc")
    allowed = re.compile(r"^(__shared__|extern __shared__|constexpr|const int|MG_IDX2|UpSmem|GreenSSmem|Green3Smem"
                         r"|T \*sm = reinterpret_cast)")
    seen = 0
    for name in ("mg_stages.cuh", "mg_fast2d.cuh", "mg_fast3d.cuh", "mg_cluster.cuh"):
        for kern, head in _kernel_heads(os.path.join(csrc, name)):
            seen += 1
            assert len(head) <= 12, (kern, head)
            for t in head:
                assert allowed.match(t), (kern, t)
                assert "[" not in t.split("=")[-1] or "__shared__" in t, (kern, t)
    assert seen >= 55


def test_every_environment_setting_is_documented_in_the_header():
    """Each environment variable the library reads is described where the
    ABI is: in include/diagmg.h."""
    import glob
    import re
    csrc = os.path.join(os.path.dirname(N.__file__), "csrc")
    read = set()
    for path in glob.glob(os.path.join(csrc, "*.cu*")):
        read |= set(re.findall(r'getenv\("([A-Z_0-9]+)"\)', open(path).read()))
    assert read, "no settings found"
    header = open(os.path.join(os.path.dirname(os.path.dirname(N.__file__)), "include", "diagmg.h")).read()
    for name in sorted(read):
        assert name in header, name


def test_python_api_surface():
    """The calls the package documents exist (no GPU needed to look them up)."""
    import inspect

    import paper_math_9907190_gb300 as P
    for name in ("Batch", "Context", "PoissonSolve", "default_omega", "solve"):
        assert hasattr(P, name), name
    for m in ("solve", "vcycle", "residual", "solve_two_stage", "set_omega", "set_sweeps", "rho", "tune",
              "tune_info", "restrict", "coarse_solve", "prolong", "level_get", "level_set", "new_grid", "close",
              "solve_host", "solve_host_many", "fp64_rate", "set_gamma"):
        assert callable(getattr(P.Context, m)), m
    for m in ("solve", "tune", "close", "statuses"):
        assert callable(getattr(P.Batch, m)), m
    assert list(inspect.signature(P.Context.__init__).parameters)[1:3] == ["dim", "n"]
    assert "from_zero" in inspect.signature(P.Context.solve).parameters
    assert P.default_omega(2, "diag", 2) == (1.052,)
