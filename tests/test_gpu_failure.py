"""Failure detection on the GPU without a GPU fault: a bounded device wait runs
out (the test hook makes the MMA issuer wait on an mbarrier that nothing
arrives on), the kernel drains, frees its tensor memory and exits, the host
reads GATTN_ERR_TIMEOUT from the status word, and the context stays usable."""
import pytest
import torch

import oracle
from paper_2604_16590_gb300 import build, gattn
from paper_2604_16590_gb300.inputs import qkv
from tests._parity import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    gattn.load_library()


def test_bounded_wait_timeout_is_reported_and_context_survives():
    grid, core, halo = (2, 32, 32), (1, 16, 16), (0, 4, 4)
    shape = (1, 2, 2 * 32 * 32, 64)
    q, k, v = (t.cuda() for t in qkv(shape, 31, 0.5, "bf16"))
    tiling = gattn.Tiling(grid, core, halo)
    desc = gattn.desc_for(q, tiling, torch.float32, flags=gattn.GATTN_FLAG_TEST_STALL)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    saved = torch.empty(gattn.gattn_saved_bytes(desc), dtype=torch.uint8, device="cuda")
    assert gattn.gattn_fwd(desc, q, k, v, out, saved) == 0
    assert gattn.gattn_stream_status() == 5  # GATTN_ERR_TIMEOUT, read from the device status word
    assert gattn.gattn_stream_status() == 0  # the word was cleared
    # the same context still computes correct results
    out2, _ = gattn.forward(q, k, v, tiling, out_dtype=torch.float32)
    assert gattn.gattn_stream_status() == 0
    geo = oracle.Geometry(1, 2, 64, *grid, core, halo)
    ref = oracle.forward(geo, *(t.double().cpu().numpy() for t in (q, k, v)))
    assert_close("after-timeout/out", out2.double().cpu().numpy(), ref, 2e-2, 3e-3)
