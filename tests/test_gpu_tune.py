"""Autotuner (mg_tune / mg_batch_tune): the tuned schedule keeps oracle parity,
the cache file is written once and reused without measuring."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_math_9907190_gb300 import Batch, Context, default_omega
from paper_math_9907190_gb300 import inputs as I
from _iterates import assert_iterate

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda", 0)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("dim,n,precision", [(2, 1023, "fp64"), (2, 1023, "mixed"), (3, 63, "fp64")])
def test_tuned_schedule_keeps_parity_and_caches(tmp_path, dim, n, precision):
    cache = str(tmp_path / "tune.jsonl")
    f = I.uniform_f(dim, n, 5) if dim == 2 else I.cube(n)
    ft = T(f)
    with Context(dim, n, precision=precision) as c:
        scratch = c.new_grid()
        assert c.tune(ft, scratch, cache=cache)
        assert float(scratch.abs().max()) == 0.0
        cut, dn, up = c.tune_info()
        assert cut in ((15, 31, 63) if dim == 2 else (7, 15))
        # FP64 levels: three tile classes; FP32 levels: three streaming strip heights and three tiles
        assert all(0 <= x < (3 if precision == "fp64" else 6) for x in dn + up)
        u, it, rel, _ = c.solve(ft, rtol=1e-10)
    assert os.path.exists(cache) and len(open(cache).read().strip().splitlines()) == 1
    with Context(dim, n, precision=precision) as c2:
        assert not c2.tune(ft, cache=cache)  # taken from the cache
        assert c2.tune_info() == (cut, dn, up)
    om = list(default_omega(dim))
    if precision == "fp64":
        uo, io, _, _ = O.solve(f, omega=om, rtol=1e-10)
        assert io == it
        assert_iterate(u.cpu().numpy(), uo, 1e-12)
    else:
        assert rel <= 1e-10


def test_batch_tune(tmp_path):
    sides = [127, 255, 127, 63]
    fs = [T(I.batch_f(n, b)) for b, n in enumerate(sides)]
    with Batch(2, sides) as bt:
        bt.tune(fs, cache=str(tmp_path / "t.jsonl"))
        us, cyc, rel = bt.solve(fs, rtol=1e-10)
    assert all(r <= 1e-10 for r in rel)
    for b, n in enumerate(sides):
        uo, _, _, _ = O.solve(fs[b].cpu().numpy(), omega=[1.052], rtol=1e-13)
        assert_iterate(us[b].cpu().numpy(), uo, 1e-8)
