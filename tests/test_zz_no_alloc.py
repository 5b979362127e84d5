"""gattn_fwd_noalloc: the forward for callers that cannot allocate device memory.

Such callers (a process whose memory manager owns all of HBM after start-up,
or a framework operator interface that hands over only inputs and outputs)
cannot supply the saved-state buffer gattn_fwd takes; this entry point keeps
that scratch in the library's own device array instead.

The test calls it through the C ABI on two problems in a row (so the second
runs on whatever the first left in the shared array) and requires each
output to equal gattn_fwd's on the same inputs bit for bit: both run the same
deterministic kernels, only the scratch address differs.  Around a call that
is not the first on the device (the first one may make the driver place the
array, under lazy module loading) it checks that nothing is allocated: the
device's free memory and torch's allocator counters are unchanged.  It also
checks that a problem too large for the array is refused before any launch.
Collected last so a failure here comes after every other test has run.
"""
import pytest
import torch

from paper_2604_16590_gb300 import build, gattn
from paper_2604_16590_gb300.inputs import qkv

pytestmark = pytest.mark.gpu

CALLS = [
    # in dtype, std, grid, core, halo
    ("bf16", 0.5, (2, 32, 32), (1, 16, 16), (0, 4, 4)),
    ("fp32", 1.0, (3, 10, 13), (2, 4, 5), (1, 2, 2)),
]

_COUNTERS = ("allocation.all.allocated", "segment.all.allocated", "num_alloc_retries", "num_device_alloc")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    gattn.load_library()


def _alloc_state(dev):
    torch.cuda.synchronize(dev)
    stats = torch.cuda.memory_stats(dev)
    return torch.cuda.mem_get_info(dev)[0], {c: stats.get(c, 0) for c in _COUNTERS}


def test_noalloc_forward_matches_gattn_fwd_on_two_calls_in_a_row():
    dev = torch.device("cuda:0")
    for n, (dt, std, grid, core, halo) in enumerate(CALLS):
        B, nh, d = 1, 2, 64
        shape = (B, nh, grid[0] * grid[1] * grid[2], d)
        q, k, v = (t.to(dev) for t in qkv(shape, 4242 + n, std, dt))
        tiling = gattn.Tiling(grid, core, halo)
        desc = gattn.desc_for(q, tiling, torch.float32)
        assert gattn.gattn_saved_bytes(desc) <= gattn.GATTN_NOALLOC_SCRATCH_BYTES
        ref = torch.empty(shape, dtype=torch.float32, device=dev)
        saved = torch.empty(gattn.gattn_saved_bytes(desc), dtype=torch.uint8, device=dev)
        gattn.check(gattn.gattn_fwd(desc, q, k, v, ref, saved), "gattn_fwd")
        out = torch.full(shape, float("nan"), dtype=torch.float32, device=dev)
        again = torch.full(shape, float("nan"), dtype=torch.float32, device=dev)
        gattn.check(gattn.gattn_fwd_noalloc(desc, q, k, v, out), "gattn_fwd_noalloc")
        st = gattn.gattn_stream_status()
        assert st == 0, gattn.STATUS.get(st, st)
        assert torch.equal(out, ref), f"call {n} ({dt}): differs from gattn_fwd"
        # a further call on the same device allocates nothing
        free0, counters0 = _alloc_state(dev)
        gattn.check(gattn.gattn_fwd_noalloc(desc, q, k, v, again), "gattn_fwd_noalloc")
        free1, counters1 = _alloc_state(dev)
        assert gattn.gattn_stream_status() == 0
        assert free1 == free0, f"device free memory moved by {free0 - free1} bytes"
        assert counters1 == counters0
        assert torch.equal(again, ref)


def test_noalloc_rejects_problems_larger_than_its_array():
    # 64 x 4 heads on a 32x64x128 grid needs far more than the array holds
    desc = gattn.make_desc(4, 16, 64, (32, 64, 128), (32, 16, 32), (0, 4, 8), in_dtype="bf16")
    assert gattn.gattn_saved_bytes(desc) > gattn.GATTN_NOALLOC_SCRATCH_BYTES
    st = gattn.gattn_fwd_noalloc(desc, 16, 16, 16, 16)
    assert st == 3  # GATTN_ERR_WORKSPACE, returned before any launch
