"""A grid whose variable planes hold more than 2^31 elements: every address
the kernels form (cells, rows, planes, halo rows, strips) has to be 64-bit.
The scheme is translation invariant, so a periodic grid tiled from a small
periodic pattern, with the same cell size, must give in every tile the bits
of the small grid run alone (its lmax, hence its dt, is the same too), with
FP32 and with bfloat16 storage."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TILE = 80
NTX, NTY = 500, 675           # 40000 x 54000 cells: 2.16e9 per plane > 2^31
STEPS = 3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def fv():
    from paper_1701_05431_gb300 import fvlib
    return fvlib


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_grid_beyond_2_31_cells_per_plane_equals_its_tile(precision):
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    # input 34.6 GB, two state buffers 69 GB (FP32), the result 34.6 GB, a comparison mask
    if free < 160e9:
        pytest.skip(f"needs about 160 GB of free device memory, {free / 1e9:.0f} GB free")
    f = fv()
    prim, d = wl.random_smooth_euler(TILE, seed=21)
    p32 = np.ascontiguousarray(prim.astype(np.float32))
    with f.Solver(d, precision) as s:
        s.set_state(p32, primitive=True)
        t_small = s.run(STEPS)
        small = torch.from_numpy(np.ascontiguousarray(s.state("float32"))).cuda()

    nx, ny = TILE * NTX, TILE * NTY
    assert nx * ny > 2 ** 31
    # the same cell size: [0, 500] x [0, 675] split into 40000 x 54000 cells
    big_d = dict(d, nx=nx, ny=ny, xmax=float(NTX), ymax=float(NTY))
    src = torch.from_numpy(p32).cuda().repeat(1, NTY, NTX)
    with f.Solver(big_d, precision) as s:
        s.set_state(src, primitive=True)
        del src
        torch.cuda.empty_cache()
        t_big = s.run(STEPS)
        out = torch.empty((4, ny, nx), dtype=torch.float32, device="cuda")
        s.get_state(out)
    assert t_big == t_small
    tiles = out.view(4, NTY, TILE, NTX, TILE)
    ref = small.view(4, 1, TILE, 1, TILE)
    for v in range(4):
        assert bool((tiles[v] == ref[v]).all()), v
    # the last column and row of tiles, which the ragged last strip and chunk hold
    assert torch.equal(out[:, -TILE:, -TILE:], small)
    del out, tiles
    torch.cuda.empty_cache()
