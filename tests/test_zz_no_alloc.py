"""gs_bin_sort_noalloc, the binning entry point for callers that cannot
allocate device memory (allocators that forbid new device allocations after
start-up, render loops that must not stall or fail on an allocation,
plug-ins handed only pre-sized buffers).  It keeps its scratch in a static
device array inside the library, so it takes no workspace.

Checked through the C ABI against gs_bin_sort with a caller workspace: the
sorted values, keys, tile ranges and pair count must be bit-identical (the
tolerance of every integer output in these tests), on two calls in a row
(the second smaller than the first, so stale scratch contents from the
first call are present).  Collected last so that a stop-at-first-failure run
has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2403_01444_gb300 import gs3, scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01444_gb300 import build
    build.build()
    gs3.lib()


def _projected(V, N, W, H, seed):
    rec = scenes.random_projected(V, N, W, H, np.random.default_rng(seed))
    t = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dt)
    p = gs3.Projected.empty(V, N, DEV)
    p.mean2d.copy_(t(rec["mean2d"]))
    p.conic_opacity.copy_(t(np.concatenate([rec["conic"], rec["opacity"][..., None]], -1)))
    p.rgb.copy_(t(rec["rgb"]))
    p.depth.copy_(t(rec["depth"]))
    p.radius.copy_(t(rec["radius"], torch.int32))
    p.tiles_touched.zero_()
    return p


def _outputs(V, N, W, H, cap):
    tiles = ((W + 15) // 16) * ((H + 15) // 16)
    z = lambda *s, dt=torch.int32: torch.zeros(*s, dtype=dt, device=DEV)
    return dict(vals=z(cap), ranges=z(V * tiles, 2), keys=z(cap, dt=torch.int64),
                count=z(1, dt=torch.int64), err=z(1))


def _run_both(V, N, W, H, seed):
    p = _projected(V, N, W, H, seed)
    cap = 200_000
    ref = _outputs(V, N, W, H, cap)
    ws = torch.empty(gs3.gs_bin_sort_workspace_size(N, V, W, H, cap), dtype=torch.uint8, device=DEV)
    gs3.gs_bin_sort(p, N, V, W, H, 1, cap, ref["vals"], ref["ranges"], ref["keys"], ref["count"],
                    ref["err"], ws)
    got = _outputs(V, N, W, H, cap)
    got["vals"].fill_(-1)
    got["keys"].fill_(-1)
    gs3.gs_bin_sort_noalloc(p, N, V, W, H, 1, cap, got["vals"], got["ranges"], got["keys"],
                            got["count"], got["err"])
    torch.cuda.synchronize()
    n = int(ref["count"].item())
    assert n > 0 and int(ref["err"].item()) == 0
    assert int(got["count"].item()) == n and int(got["err"].item()) == 0
    assert torch.equal(got["vals"][:n], ref["vals"][:n])
    assert torch.equal(got["keys"][:n], ref["keys"][:n])
    assert torch.equal(got["ranges"], ref["ranges"])


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    _run_both(3, 4000, 300, 200, 1)   # first call
    _run_both(2, 900, 130, 90, 2)     # second, smaller call over the first call's scratch


def test_noalloc_rejects_oversized_problems():
    V, W, H = 1, 64, 64
    p = _projected(V, 8, W, H, 3)
    o = _outputs(V, 8, W, H, 16)
    with pytest.raises(gs3.GsError) as e:
        # n * V above the 131072-entry limit: refused before any launch
        gs3.gs_bin_sort_noalloc(p, 200_000, V, W, H, 1, 16, o["vals"], o["ranges"], o["keys"],
                                o["count"], o["err"])
    assert e.value.status == gs3.GS_ERR_INVALID_ARG
    with pytest.raises(gs3.GsError) as e:
        gs3.gs_bin_sort_noalloc(p, 8, V, W, H, 1, 1 << 21, o["vals"], o["ranges"], o["keys"],
                                o["count"], o["err"])
    assert e.value.status == gs3.GS_ERR_INVALID_ARG
