"""Failure detection on the GPU without a fault: the tensor-core kernels'
bounded mbarrier wait, made to run out on a barrier nothing arrives on,
returns a timeout status the host reads, and the context stays usable."""
import time

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


def test_bounded_wait_times_out_and_context_stays_usable():
    status = torch.full((1,), 12345, dtype=torch.int32, device=DEV)
    t0 = time.perf_counter()
    gs3.gs_tc_wait_selftest(4096, status)
    torch.cuda.synchronize()
    assert int(status.item()) == gs3.GS_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    # the context still runs the tensor-core MLP, with the result of the FP32 path
    rng = np.random.default_rng(5)
    n = 1000
    enc = torch.from_numpy(rng.integers(-2, 3, size=(n, 32)).astype(np.float32)).to(DEV)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    w = np.concatenate([(np.round(x * 8) / 8).ravel() for x in Ws]).astype(np.float32)  # exact in BF16
    w32 = torch.from_numpy(w).to(DEV)
    wbf = w32.to(torch.bfloat16)
    out_tc = torch.zeros(n, 7, device=DEV)
    out_32 = torch.zeros(n, 7, device=DEV)
    gs3.ntc_mlp_fwd(enc.to(torch.bfloat16), n, gs3.mlp_struct(gs3.GS_MLP_BF16, w32, wbf), out_tc)
    gs3.ntc_mlp_fwd(enc, n, gs3.mlp_struct(gs3.GS_MLP_FP32, w32), out_32)
    torch.cuda.synchronize()
    scale = float(out_32.abs().max())
    assert float((out_tc - out_32).abs().max()) <= 1e-2 * max(scale, 1.0)
