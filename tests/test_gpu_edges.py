"""Edge cases of the solve through the C ABI: the smallest grids in mixed
precision, caller arrays with a padded row pitch (the padding is neither
read into the result nor written), the launch settings (programmatic
dependent launch on, off, or on small grids only) giving the same bits, and
misaligned grid pointers refused before any launch."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_math_9907190_gb300 import Context, default_omega
from paper_math_9907190_gb300 import inputs as I
from _iterates import assert_iterate

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda", 0)


def _f(dim, n, seed=1):
    return I.uniform_f(dim, n, seed) if dim == 2 else I.cube(n)


def _check_against_oracle(dim, n, f, u, rel, order=2):
    """Final relative residual by the oracle, and the solution against the
    oracle's converged FP64 solution."""
    assert rel <= 1e-10
    r = O.residual(f, u, order)
    r0 = O.residual(f, O.grid(dim, n), order)
    assert math.sqrt(O.norm2_interior(r) / O.norm2_interior(r0)) <= 1.05e-10
    uo, _, _, _ = O.solve(f, omega=list(default_omega(dim, "diag", order)), rtol=1e-13, max_cycles=200)
    assert_iterate(u, uo, 1e-8)


@pytest.mark.parametrize("dim,n", [(2, 3), (2, 7), (2, 15), (3, 3), (3, 7), (3, 15)])
def test_smallest_grids_mixed(dim, n):
    """Grids with one to three levels above the coarsest: every level runs in
    the single coarse thread block."""
    f = _f(dim, n)
    with Context(dim, n, precision="mixed", omega=default_omega(dim, "diag", 2)) as c:
        u, it, rel, hist = c.solve(torch.from_numpy(f).to(DEV), rtol=1e-10, max_cycles=40)
    assert 1 <= it <= 12 and len(hist) == it
    _check_against_oracle(dim, n, f, u.cpu().numpy(), rel)


def _padded(a, pitch, fill):
    """A device copy of the full grid `a` inside rows of `pitch` elements; the
    columns beyond n + 2 hold `fill`.  Returns (view, backing tensor)."""
    shape = a.shape[:-1] + (pitch,)
    back = torch.full(shape, fill, dtype=torch.float64, device=DEV)
    view = back[..., : a.shape[-1]]
    view.copy_(torch.from_numpy(a))
    return view, back


@pytest.mark.parametrize("dim,n,pad", [(2, 255, 45), (2, 1023, 7), (3, 31, 6), (3, 63, 11)])
def test_padded_pitch_solve_leaves_padding_alone(dim, n, pad):
    """The fused mixed path (carried residual) with a caller pitch above n + 2:
    the padding holds NaN, which must neither reach the result nor be
    overwritten."""
    f = _f(dim, n)
    pitch = n + 2 + pad
    fv, fb = _padded(f, pitch, float("nan"))
    uv, ub = _padded(np.zeros_like(f), pitch, float("nan"))
    with Context(dim, n, precision="mixed", omega=default_omega(dim, "diag", 2), pitch=pitch) as c:
        _, it, rel, _ = c.solve(fv, uv, rtol=1e-10, max_cycles=40)
    assert torch.isnan(ub[..., n + 2:]).all() and torch.isnan(fb[..., n + 2:]).all()
    u = uv.cpu().numpy()
    assert np.isfinite(u).all()
    ring = np.ones(u.shape, dtype=bool)
    ring[(slice(1, -1),) * dim] = False
    assert (u[ring] == 0.0).all()
    # the same solve on unpadded arrays gives the same bits
    with Context(dim, n, precision="mixed", omega=default_omega(dim, "diag", 2)) as c:
        u2, it2, rel2, _ = c.solve(torch.from_numpy(f).to(DEV), rtol=1e-10, max_cycles=40)
    assert it2 == it and rel2 == rel
    assert np.array_equal(u2.cpu().numpy(), u)
    _check_against_oracle(dim, n, f, u, rel)


@pytest.mark.parametrize("dim,n,prec", [(2, 255, "mixed"), (3, 31, "mixed"), (2, 127, "fp64")])
def test_padded_pitch_solve_from_zero_leaves_padding_alone(dim, n, prec):
    """mg_solve_zero zeroes u itself: its (n+2)^d points only, not the
    padding of a larger caller pitch (which holds NaN here), and with the same
    bits as the unpadded solve."""
    f = _f(dim, n)
    pitch = n + 2 + 5
    fv, fb = _padded(f, pitch, float("nan"))
    uv, ub = _padded(np.full_like(f, 3.0), pitch, float("nan"))
    with Context(dim, n, precision=prec, omega=default_omega(dim, "diag", 2), pitch=pitch) as c:
        _, it, rel, _ = c.solve(fv, uv, rtol=1e-10, max_cycles=40, from_zero=True)
    assert torch.isnan(ub[..., n + 2:]).all() and torch.isnan(fb[..., n + 2:]).all()
    with Context(dim, n, precision=prec, omega=default_omega(dim, "diag", 2)) as c:
        u2, it2, rel2, _ = c.solve(torch.from_numpy(f).to(DEV), rtol=1e-10, max_cycles=40)
    assert it2 == it and rel2 == rel
    assert np.array_equal(u2.cpu().numpy(), uv.cpu().numpy())


@pytest.mark.parametrize("dim,n,prec", [(2, 1023, "mixed"), (2, 255, "fp64"), (3, 63, "mixed"), (3, 31, "fp64")])
def test_launch_settings_give_the_same_bits(dim, n, prec, monkeypatch):
    """Programmatic dependent launch changes when a kernel is scheduled, never
    what it computes: every kernel waits for the previous one before its first
    access to memory."""
    f = torch.from_numpy(_f(dim, n)).to(DEV)
    outs = []
    for pdl, maxb in (("0", "0"), ("1", "0"), ("1", "64")):
        monkeypatch.setenv("DIAGMG_PDL", pdl)
        monkeypatch.setenv("DIAGMG_PDL_MAX_BLOCKS", maxb)
        with Context(dim, n, precision=prec, omega=default_omega(dim, "diag", 2)) as c:
            u, it, rel, hist = c.solve(f, rtol=1e-10, max_cycles=40)
            c.vcycle(f, u)  # the per-cycle entry point too
            outs.append((u.cpu().numpy(), it, rel, hist))
    for u, it, rel, hist in outs[1:]:
        assert it == outs[0][1] and rel == outs[0][2] and hist == outs[0][3]
        assert np.array_equal(u, outs[0][0])


def test_misaligned_grid_pointers_are_refused_before_any_launch():
    """A grid pointer off an FP64 element boundary is an argument error: the
    call returns MG_EINVAL and launches nothing."""
    import ctypes

    from paper_math_9907190_gb300 import _native as N

    n = 63
    with Context(2, n, precision="mixed") as c:
        f = torch.from_numpy(_f(2, n)).to(DEV)
        u = c.new_grid()
        lib = N.lib()
        before = c.launch_count()
        ok, bad = ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr() + 4)
        fp = ctypes.c_void_p(f.data_ptr())
        cyc, rel = ctypes.c_int(), ctypes.c_double()
        assert lib.mg_solve(c._h, fp, bad, 1e-10, 10, ctypes.byref(cyc), ctypes.byref(rel), None, None) == N.MG_EINVAL
        assert lib.mg_solve(c._h, ctypes.c_void_p(f.data_ptr() + 2), ok, 1e-10, 10, None, None, None,
                            None) == N.MG_EINVAL
        assert lib.mg_vcycle(c._h, fp, bad, None) == N.MG_EINVAL
        assert lib.mg_residual(c._h, fp, bad, ctypes.c_double(1.0 / (n + 1)), 2, None, None, None) == N.MG_EINVAL
        assert lib.mg_level_get(c._h, 0, 0, bad, None) == N.MG_EINVAL
        assert c.launch_count() == before
        # the same context still solves
        _, it, rel2, _ = c.solve(f, u, rtol=1e-10, max_cycles=40)
        assert rel2 <= 1e-10


@pytest.mark.parametrize("dim,n,omega", [(2, 63, (1.052,)), (2, 255, (1.3,)), (3, 15, (1.11, 1.42, 1.08, 0.99)),
                                         (3, 31, (0.9, 1.2, 1.3, 1.25))])
def test_odd_point_errors_are_scaled_by_one_minus_p(dim, n, omega):
    """An error supported on the finest grid's odd-index-sum points has a zero
    restricted residual (the first restriction weights a point 2d times each
    axis neighbour), so every coarse correction vanishes and the final
    half-sweeps return exactly (1 - p) e, p the finest weight (p_g in 3D).
    The FP64 cycle on the GPU meets this to rounding."""
    rng = np.random.default_rng(19)
    idx = np.indices((n + 2,) * dim)
    inner = np.zeros((n + 2,) * dim, dtype=bool)
    inner[(slice(1, -1),) * dim] = True
    e = np.where(inner & (idx.sum(0) % 2 == 1), rng.standard_normal((n + 2,) * dim), 0.0)
    with Context(dim, n, precision="fp64", omega=omega) as c:
        u = torch.from_numpy(e.copy()).to(DEV)
        c.vcycle(torch.zeros_like(u), u)
        got = u.cpu().numpy()
    assert np.abs(got - (1.0 - omega[-1]) * e).max() <= 1e-12 * np.abs(e).max()
