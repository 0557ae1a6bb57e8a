"""Python API over the C ABI: contexts, solves and the autograd adjoint.

PyTorch supplies device memory and streams only; every step of the method
runs in the CUDA kernels of libdiagmg.so.  Arrays are CUDA float64 tensors
holding the full grid (Dirichlet ring included), shape (n+2,)*dim, x the last
(fastest) axis.
"""

from __future__ import annotations

import ctypes

import torch

from . import _native as N

# Over-relaxation weights the paper found optimal (Table 1: 2D p; Table 3:
# 3D p_m, p_r1, p_r2, p_g for the diagonal cycle and p_g for the usual one).
PAPER_OMEGA = {
    (2, "diag", 2): (1.052,), (2, "diag", 4): (1.2,),
    (2, "usual", 2): (1.121,), (2, "usual", 4): (1.216,),
    (3, "diag", 2): (1.11, 1.42, 1.08, 0.99), (3, "diag", 4): (0.91, 0.80, 0.70, 1.77),
    (3, "usual", 2): (1.30,), (3, "usual", 4): (1.70,),
}


def default_omega(dim: int, hierarchy: str = "diag", order: int = 2) -> tuple:
    return PAPER_OMEGA[(dim, hierarchy, order)]


def _hier(h):
    return {"diag": N.MG_DIAG, "usual": N.MG_USUAL}[h]


def _prec(p):
    return {"fp64": N.MG_FP64, "mixed": N.MG_MIXED}[p]


class Context:
    """One solver context (mg_create) for a fixed grid, hierarchy, order and precision."""

    def __init__(self, dim: int, n: int, *, hierarchy: str = "diag", order: int = 2, precision: str = "fp64",
                 coarsest: int = 3, omega=None, pitch: int | None = None, device=None):
        self.dim, self.n, self.order = dim, n, order
        self.hierarchy, self.precision = hierarchy, precision
        self.pitch = n + 2 if pitch is None else pitch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        om = tuple(default_omega(dim, hierarchy, order) if omega is None else omega)
        self.omega = om
        d = N.mg_desc()
        d.dim, d.n, d.pitch = dim, n, self.pitch
        d.hierarchy, d.order, d.precision, d.coarsest = _hier(hierarchy), order, _prec(precision), coarsest
        for i in range(4):
            d.omega[i] = om[i] if i < len(om) else 1.0
        self._desc = d
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            N.check(N.lib().mg_create(ctypes.byref(self._h), ctypes.byref(d)), "mg_create")
        nl = ctypes.c_int()
        N.check(N.lib().mg_num_levels(self._h, ctypes.byref(nl)), "mg_num_levels")
        self.num_levels = nl.value

    # -- plumbing ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            N.lib().mg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _grid(self, t: torch.Tensor, name: str):
        n, dim = self.n, self.dim
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float64:
            raise TypeError(f"{name}: expected a CUDA float64 tensor")
        if t.dim() != dim or tuple(t.shape) != (n + 2,) * dim:
            raise ValueError(f"{name}: expected shape {(n + 2,) * dim}, got {tuple(t.shape)}")
        want = (self.pitch,) if dim == 2 else (self.pitch * (n + 2), self.pitch)
        if t.stride(-1) != 1 or tuple(t.stride()[:-1]) != want:
            raise ValueError(f"{name}: strides {t.stride()} do not match pitch {self.pitch}")
        return ctypes.c_void_p(t.data_ptr())

    def new_grid(self) -> torch.Tensor:
        return torch.zeros((self.n + 2,) * self.dim, dtype=torch.float64, device=self.device)

    def level_info(self, level: int):
        s, k = ctypes.c_int(), ctypes.c_int()
        N.check(N.lib().mg_level_info(self._h, level, ctypes.byref(s), ctypes.byref(k)), "mg_level_info")
        return s.value, k.value

    # -- diagnostics ---------------------------------------------------------
    def launch_count(self) -> int:
        v = ctypes.c_longlong()
        N.check(N.lib().mg_launch_count(self._h, ctypes.byref(v)), "mg_launch_count")
        return v.value

    def probe_set(self, family: int):
        N.check(N.lib().mg_probe_set(self._h, family), "mg_probe_set")

    def probe_read(self):
        """(launches, total ms) of the probed kernel family since probe_set."""
        n, ms = ctypes.c_longlong(), ctypes.c_double()
        N.check(N.lib().mg_probe_read(self._h, ctypes.byref(n), ctypes.byref(ms), self._stream()), "mg_probe_read")
        return n.value, ms.value

    def solve_two_stage(self, f, u=None, *, omega2=None, rtol2: float = 1e-4, rtol: float = 1e-10,
                        max_cycles: int = 100, raise_on_fail: bool = True):
        """mg_solve_two_stage (order-4 context): second-order V-cycles to rtol2,
        then fourth-order cycles to rtol.  Returns (u, cycles2, cycles4, relres)."""
        if self.order != 4:
            raise ValueError("two-stage solves need an order-4 context")
        u = self.new_grid() if u is None else u
        om2 = default_omega(self.dim, self.hierarchy, 2) if omega2 is None else omega2
        arr = (ctypes.c_double * 4)(*(list(om2) + [1.0] * (4 - len(om2))))
        c2, c4, rel = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        st = N.lib().mg_solve_two_stage(self._h, self._grid(f, "f"), self._grid(u, "u"), arr, rtol2, rtol, max_cycles,
                                        ctypes.byref(c2), ctypes.byref(c4), ctypes.byref(rel), self._stream())
        if raise_on_fail:
            N.check(st, "mg_solve_two_stage")
        return u, c2.value, c4.value, rel.value

    def solve_host(self, f, u=None, *, u0=None, rtol: float = 1e-10, max_cycles: int = 100,
                   raise_on_fail: bool = True):
        """mg_solve_host: f, u0 (warm start; None: u = 0) and u (the result;
        default a new tensor) are CPU float64 full grids -- pin them for full
        copy bandwidth.  Returns (u, cycles, relres)."""
        shape = (self.n + 2,) * (self.dim - 1) + (self.pitch,)
        u = torch.empty(shape, dtype=torch.float64) if u is None else u
        for name, t in (("f", f), ("u", u), ("u0", u0)):
            if t is None:
                continue
            if t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != shape:
                raise ValueError(f"{name}: expected a contiguous CPU float64 tensor of shape {shape}")
        cyc, rel = ctypes.c_int(), ctypes.c_double()
        st = N.lib().mg_solve_host(self._h, ctypes.c_void_p(f.data_ptr()),
                                   ctypes.c_void_p(u0.data_ptr()) if u0 is not None else None,
                                   ctypes.c_void_p(u.data_ptr()), rtol, max_cycles, ctypes.byref(cyc),
                                   ctypes.byref(rel), self._stream())
        if raise_on_fail:
            N.check(st, "mg_solve_host")
        return u, cyc.value, rel.value

    def solve_host_many(self, fs, us=None, *, rtol: float = 1e-10, max_cycles: int = 100,
                        raise_on_fail: bool = True):
        """mg_solve_host_many: each f in fs (CPU float64 full grids, pinned for
        full copy bandwidth) solved from u = 0 into the matching u of us
        (default new tensors), copies and solves pipelined.  Returns (us,
        cycles, relres) with per-problem lists."""
        shape = (self.n + 2,) * (self.dim - 1) + (self.pitch,)
        us = [torch.empty(shape, dtype=torch.float64) for _ in fs] if us is None else us
        if len(us) != len(fs):
            raise ValueError("fs and us differ in length")
        for name, ts in (("f", fs), ("u", us)):
            for t in ts:
                if t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != shape:
                    raise ValueError(f"{name}: expected contiguous CPU float64 tensors of shape {shape}")
        k = len(fs)
        fp = (ctypes.c_void_p * max(1, k))(*[t.data_ptr() for t in fs])
        up = (ctypes.c_void_p * max(1, k))(*[t.data_ptr() for t in us])
        cyc = (ctypes.c_int * max(1, k))()
        rel = (ctypes.c_double * max(1, k))()
        st = N.lib().mg_solve_host_many(self._h, k, fp, up, rtol, max_cycles, cyc, rel, self._stream())
        if raise_on_fail:
            N.check(st, "mg_solve_host_many")
        return us, list(cyc)[:k], list(rel)[:k]

    def fp64_rate(self) -> float:
        """mg_fp64_rate: measured FP64 pipe operations per second of this device."""
        v = ctypes.c_double()
        N.check(N.lib().mg_fp64_rate(self._h, ctypes.byref(v), self._stream()), "mg_fp64_rate")
        return v.value

    def set_omega(self, omega):
        """mg_set_omega: new over-relaxation weights for later cycles."""
        arr = (ctypes.c_double * 4)(*(list(omega) + [1.0] * (4 - len(omega))))
        N.check(N.lib().mg_set_omega(self._h, arr), "mg_set_omega")
        self.omega = tuple(omega)

    def set_gamma(self, gamma: int):
        """mg_set_gamma: gamma cycles of each coarse problem per visit (2D
        diagonal; 1 is the V-cycle, 2 the W-cycle)."""
        N.check(N.lib().mg_set_gamma(self._h, gamma), "mg_set_gamma")

    def set_sweeps(self, extra: int):
        """mg_set_sweeps: extra Jacobi sweeps per level (2D diagonal hierarchy)."""
        N.check(N.lib().mg_set_sweeps(self._h, int(extra)), "mg_set_sweeps")
        self.extra = int(extra)

    def rho(self, cycles: int = 60, skip: int = 40, seed: int = 0) -> float:
        """mg_rho: convergence factor of the V-cycle by power iteration from a
        seeded random start (interior U[-1, 1])."""
        g = torch.Generator(device="cpu").manual_seed(seed)
        u = torch.rand((self.n + 2,) * self.dim, generator=g, dtype=torch.float64) * 2 - 1
        ring = torch.ones_like(u, dtype=torch.bool)
        ring[(slice(1, -1),) * self.dim] = False
        u[ring] = 0.0
        u = u.to(self.device)
        z = torch.zeros_like(u)
        out = ctypes.c_double()
        N.check(N.lib().mg_rho(self._h, self._grid(z, "zero_f"), self._grid(u, "u"), cycles, skip, ctypes.byref(out),
                               self._stream()), "mg_rho")
        return out.value

    def tune(self, f, u=None, cache: str | None = None) -> bool:
        """mg_tune: measure (or take from the cache file) the coarse-block
        cut-off and the tile shape of every pair kernel; u is scratch, left 0.
        Returns True when it measured."""
        u = self.new_grid() if u is None else u
        measured = ctypes.c_int()
        N.check(N.lib().mg_tune(self._h, self._grid(f, "f"), self._grid(u, "u"),
                                cache.encode() if cache else None, ctypes.byref(measured), self._stream()), "mg_tune")
        return bool(measured.value)

    def tune_info(self):
        """(cut-off side (0 = default), tile classes of the down kernels, of the up kernels)."""
        cut, npair = ctypes.c_int(), ctypes.c_int()
        dn, upv = (ctypes.c_int * 32)(), (ctypes.c_int * 32)()
        N.check(N.lib().mg_tune_info(self._h, ctypes.byref(cut), ctypes.byref(npair), dn, upv), "mg_tune_info")
        return cut.value, list(dn[: npair.value]), list(upv[: npair.value])

    # -- the C ABI, one method per call ------------------------------------
    def residual(self, f, u, r=None, norm: bool = True):
        """mg_residual: returns sum(r^2) (float) when norm, else None."""
        out = ctypes.c_double()
        rp = self._grid(r, "r") if r is not None else None
        N.check(N.lib().mg_residual(self._h, self._grid(f, "f"), self._grid(u, "u"), 1.0 / (self.n + 1),
                                    self.order, rp, ctypes.byref(out) if norm else None, self._stream()),
                "mg_residual")
        return out.value if norm else None

    def restrict(self, level: int):
        N.check(N.lib().mg_restrict_diag(self._h, level, self._stream()), "mg_restrict_diag")

    def coarse_solve(self):
        N.check(N.lib().mg_coarse_solve(self._h, self._stream()), "mg_coarse_solve")

    def prolong(self, level: int, omega=None):
        om = None
        if omega is not None:
            arr = (ctypes.c_double * 4)(*(list(omega) + [1.0] * (4 - len(omega))))
            om = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        N.check(N.lib().mg_jacobi_prolong(self._h, level, om, self._stream()), "mg_jacobi_prolong")

    def level_get(self, level: int, which: str = "r", out: torch.Tensor | None = None) -> torch.Tensor:
        side, _ = self.level_info(level)
        g = torch.zeros((side + 2,) * self.dim, dtype=torch.float64, device=self.device) if out is None else out
        N.check(N.lib().mg_level_get(self._h, level, {"r": 0, "v": 1}[which], ctypes.c_void_p(g.data_ptr()),
                                     self._stream()), "mg_level_get")
        return g

    def level_set(self, level: int, which: str, grid: torch.Tensor):
        side, _ = self.level_info(level)
        assert grid.is_contiguous() and grid.dtype == torch.float64 and tuple(grid.shape) == (side + 2,) * self.dim
        N.check(N.lib().mg_level_set(self._h, level, {"r": 0, "v": 1}[which], ctypes.c_void_p(grid.data_ptr()),
                                     self._stream()), "mg_level_set")

    def vcycle(self, f, u):
        N.check(N.lib().mg_vcycle(self._h, self._grid(f, "f"), self._grid(u, "u"), self._stream()), "mg_vcycle")
        return u

    def solve(self, f, u=None, *, rtol: float = 1e-10, max_cycles: int = 100, raise_on_fail: bool = True,
              from_zero: bool = False):
        """mg_solve from the warm start u, or mg_solve_zero (from u = 0; u is
        output only) when from_zero or when u is None (a new grid).  Returns
        (u, cycles, relres, history)."""
        if u is None:
            u = torch.empty((self.n + 2,) * self.dim, dtype=torch.float64, device=self.device)
            from_zero = True
        cyc, rel = ctypes.c_int(), ctypes.c_double()
        hist = (ctypes.c_double * max(1, max_cycles))()
        name = "mg_solve_zero" if from_zero else "mg_solve"
        st = getattr(N.lib(), name)(self._h, self._grid(f, "f"), self._grid(u, "u"), rtol, max_cycles,
                                    ctypes.byref(cyc), ctypes.byref(rel), hist, self._stream())
        if raise_on_fail:
            N.check(st, name)
        return u, cyc.value, rel.value, list(hist[: cyc.value])


class Batch:
    """Many independent problems solved together (mg_batch_create / mg_solve_batched).

    sides: interior side n_b = 2^k - 1 of every problem.  Problems of equal
    side share kernel launches; the whole batched solve is one graph launch."""

    def __init__(self, dim: int, sides, *, hierarchy: str = "diag", precision: str = "mixed", coarsest: int = 3,
                 omega=None, device=None):
        self.dim, self.sides = dim, [int(x) for x in sides]
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        om = tuple(default_omega(dim, hierarchy, 2) if omega is None else omega)
        arr = (ctypes.c_double * 4)(*(list(om) + [1.0] * (4 - len(om))))
        ns = (ctypes.c_int * len(self.sides))(*self.sides)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            N.check(N.lib().mg_batch_create(ctypes.byref(self._h), dim, len(self.sides), ns, _hier(hierarchy), 2,
                                            _prec(precision), coarsest, arr), "mg_batch_create")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            N.lib().mg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def launch_count(self) -> int:
        v = ctypes.c_longlong()
        N.check(N.lib().mg_batch_launch_count(self._h, ctypes.byref(v)), "mg_batch_launch_count")
        return v.value

    def statuses(self):
        """mg_batch_status: per problem of the last solve, MG_OK, MG_ENOCONV or MG_EDIVERGED."""
        st = (ctypes.c_int * len(self.sides))()
        N.check(N.lib().mg_batch_status(self._h, st), "mg_batch_status")
        return list(st)

    def tune(self, fs, us=None, cache: str | None = None):
        """mg_batch_tune: tune every size group (us are scratch, left zero)."""
        nb = len(self.sides)
        us = [torch.zeros_like(f) for f in fs] if us is None else us
        fp = (ctypes.c_void_p * nb)(*[f.data_ptr() for f in fs])
        up = (ctypes.c_void_p * nb)(*[u.data_ptr() for u in us])
        stream = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        N.check(N.lib().mg_batch_tune(self._h, fp, up, cache.encode() if cache else None, stream), "mg_batch_tune")
        return us

    def solve(self, fs, us=None, *, rtol: float = 1e-10, max_cycles: int = 100, raise_on_fail: bool = True):
        """fs: list of CUDA float64 full grids; us: warm starts (default zeros).
        Returns (us, cycles, relres) with per-problem lists."""
        nb = len(self.sides)
        assert len(fs) == nb
        if us is None:
            us = [torch.zeros_like(f) for f in fs]
        for f, u, n in zip(fs, us, self.sides):
            for t in (f, u):
                if t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != (n + 2,) * self.dim:
                    raise ValueError("batch arrays must be contiguous float64 full grids of side n+2")
        fp = (ctypes.c_void_p * nb)(*[f.data_ptr() for f in fs])
        up = (ctypes.c_void_p * nb)(*[u.data_ptr() for u in us])
        cyc = (ctypes.c_int * nb)()
        rel = (ctypes.c_double * nb)()
        stream = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        st = N.lib().mg_solve_batched(self._h, fp, up, rtol, max_cycles, cyc, rel, stream)
        if raise_on_fail:
            N.check(st, "mg_solve_batched")
        return us, list(cyc), list(rel)


_CTX_CACHE: dict = {}


def _ctx(dim, n, hierarchy, order, precision, coarsest, omega, device):
    key = (dim, n, hierarchy, order, precision, coarsest, tuple(omega) if omega else None, str(device))
    c = _CTX_CACHE.get(key)
    if c is None:
        c = Context(dim, n, hierarchy=hierarchy, order=order, precision=precision, coarsest=coarsest,
                    omega=omega, device=device)
        _CTX_CACHE[key] = c
    return c


def solve(f: torch.Tensor, *, order: int = 2, hierarchy: str = "diag", precision: str = "mixed",
          rtol: float = 1e-10, max_cycles: int = 100, coarsest: int = 3, omega=None, u0=None):
    """Solve Laplacian(u) = f (zero Dirichlet ring) on the unit square / cube.

    f: CUDA float64 full grid (n+2,)*dim.  Returns (u, info) with info a dict
    holding cycles, relres and the residual history."""
    dim, n = f.dim(), f.shape[0] - 2
    c = _ctx(dim, n, hierarchy, order, precision, coarsest, omega, f.device)
    u = u0.clone() if u0 is not None else None
    u, cyc, rel, hist = c.solve(f.contiguous(), u, rtol=rtol, max_cycles=max_cycles)
    return u, {"cycles": cyc, "relres": rel, "history": hist}


_BATCH_CACHE: dict = {}


def _batch(dim, sides, precision, device):
    key = (dim, tuple(sides), precision, str(device))
    b = _BATCH_CACHE.get(key)
    if b is None:
        b = Batch(dim, sides, precision=precision, device=device)
        _BATCH_CACHE[key] = b
    return b


def _solve_any(f, rtol, precision, max_cycles):
    """Solve one problem (f: (n+2,)*dim, dim 2 or 3) or a stack of 3D problems
    of one size (f: (B, n+2, n+2, n+2)) as one batch."""
    if f.dim() == 4:
        dim = f.dim() - 1
        nb, n = f.shape[0], f.shape[1] - 2
        bt = _batch(dim, [n] * nb, precision, f.device)
        fs = [f[b].contiguous() for b in range(nb)]
        us = [torch.zeros_like(x) for x in fs]
        us, _, _ = bt.solve(fs, us, rtol=rtol, max_cycles=max_cycles)
        return torch.stack(us)
    u, _ = solve(f, order=2, precision=precision, rtol=rtol, max_cycles=max_cycles)
    return u


def _interior_only(g):
    g = g.contiguous().clone()
    ring = torch.ones(g.shape[-3:] if g.dim() == 4 else g.shape, dtype=torch.bool, device=g.device)
    ring[(slice(1, -1),) * ring.dim()] = False
    g[..., ring] = 0.0
    return g


class PoissonSolve(torch.autograd.Function):
    """u = L^-1 f for the discrete Dirichlet Laplacian, differentiable in f.

    f: one full grid (n+2,)*dim, or a stack (B, n+2, n+2, n+2) of 3D problems.
    Forward: multigrid solves to `rtol`.  Backward: L is symmetric under
    homogeneous Dirichlet data, so the adjoint of the solve is the same solve
    applied to the incoming gradient, grad_f = L^-1 grad_u on the interior (the
    ring of f is not read by the second-order operator, so its gradient is 0)."""

    @staticmethod
    def forward(ctx, f, rtol=1e-10, precision="mixed", max_cycles=100):
        ctx.cfg = (rtol, precision, max_cycles)
        return _solve_any(f, rtol, precision, max_cycles)

    @staticmethod
    def backward(ctx, g):
        rtol, precision, max_cycles = ctx.cfg
        w = _solve_any(_interior_only(g), rtol, precision, max_cycles)
        return w, None, None, None
