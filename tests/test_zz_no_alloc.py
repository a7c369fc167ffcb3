"""fv_totals_noalloc: the conservation totals for callers that cannot let the
library allocate device memory (loops that forbid allocator calls, frameworks
that own all device memory).  It must return what the allocating entry point
fv_totals returns, call after call, while keeping its partial sums in the
library's fixed device array.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test; it passes alone in a fresh
process too."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_totals_noalloc_matches_fv_totals_twice(precision):
    from paper_1701_05431_gb300 import fvlib
    prim, d = wl.random_smooth_euler(301, seed=29, ny=187)
    stream = torch.cuda.current_stream().cuda_stream
    dtype = torch.float64 if precision == "f64" else torch.float32
    with fvlib.Solver(d, precision, stream=stream) as s:
        s.set_state(prim, primitive=True)
        s.run(17)
        expect = s.totals()                                  # allocating entry point
        state = torch.empty((4, 187, 301), dtype=dtype, device="cuda")
        s.get_state(state)                                   # caller-owned device state
    scale = np.abs(state.double().cpu().numpy()).sum(axis=(1, 2)) / (301 * 187)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):                                    # two calls in a row share the scratch
        out.fill_(float("nan"))
        st = fvlib.totals_noalloc(state, out, (1.0 / 301) * (1.0 / 187), stream)
        assert st == fvlib.FV_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - expect) <= 1e-15 * scale), (call, got, expect)


def test_totals_noalloc_rejects_more_variables_than_its_scratch_holds():
    from paper_1701_05431_gb300 import fvlib
    state = torch.zeros((9, 4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros((9,), dtype=torch.float64, device="cuda")
    assert fvlib.totals_noalloc(state, out, 1.0) == fvlib.FV_ERR_INVALID_ARG
    assert b"8" in fvlib.load().fv_last_error(None)
