"""The C-ABI library loads on a machine without a GPU, exports every entry
point include/gattn.h declares, and validates descriptors on the host."""
import ctypes
import os
import re

import pytest

from paper_2604_16590_gb300 import build, gattn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gattn.load_library()


def _declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gattn_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_entry_point(lib):
    names = _declared_functions()
    assert "gattn_fwd" in names and "gattn_bwd" in names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_abi_version_and_status_strings(lib):
    assert gattn.gattn_abi_version() == 1
    for code in gattn.STATUS:
        assert gattn.gattn_status_string(code)


def _desc(**kw):
    base = dict(B=2, nh=3, d=64, grid=(4, 16, 32), core=(2, 8, 8), halo=(1, 2, 2), in_dtype="bf16")
    base.update(kw)
    return gattn.make_desc(**base)


def test_validate_and_sizes(lib):
    d = _desc()
    assert gattn.gattn_validate(d) == 0
    assert gattn.gattn_num_tiles(d) == 2 * 2 * 4
    # Lmax = 4 (t: [0,3),[1,4) clip ->3? ) computed independently below
    T, Y, X = 4, 16, 32
    def emax(G, c, h):
        return max(min((k + 1) * c + h, G) - max(k * c - h, 0) for k in range(-(-G // c)))
    Lmax = emax(T, 2, 1) * emax(Y, 8, 2) * emax(X, 8, 2)
    S = 2 * 3 * 16 * Lmax
    assert gattn.gattn_saved_bytes(d) >= S * 4 + S * 64 * 4
    assert gattn.gattn_bwd_workspace_bytes(d) >= 2 * S * 4 + 3 * S * 64 * 4


@pytest.mark.parametrize(
    "kw",
    [dict(d=48), dict(d=32), dict(B=0), dict(core=(0, 8, 8)), dict(halo=(-1, 0, 0)), dict(in_dtype="fp32", d=96), dict(window="hann", scale=-1.0)],
)
def test_invalid_descriptors_rejected(lib, kw):
    d = _desc(**kw)
    assert gattn.gattn_validate(d) == 1
    assert gattn.gattn_saved_bytes(d) == 0
    assert gattn.gattn_num_tiles(d) == -1


@pytest.mark.parametrize(
    "kw,ok",
    [
        # one tile as long as 32-bit slot indices allow: 2^24 - 1 boxes of 128 rows
        (dict(B=1, nh=1, grid=(1, 1, 2**31 - 129), core=(1, 1, 2**31 - 129), halo=(0, 0, 0)), True),
        (dict(B=1, nh=1, grid=(1, 2, 2**30 - 1), core=(1, 2, 2**30 - 1), halo=(0, 0, 0)), False),  # 2^24 boxes
        (dict(B=1, nh=1, grid=(1, 1, 2**31 - 1), core=(1, 1, 2**31 - 1), halo=(0, 0, 0)), False),
        (dict(B=1, nh=1, grid=(1, 1, 2**31 - 1), core=(1, 1, 1), halo=(0, 0, 0)), False),  # 2^31 - 1 tiles
        (dict(B=1, nh=1, grid=(1, 2, 2**30), core=(1, 1, 2**30), halo=(0, 0, 0)), False),  # N = 2^31
        (dict(B=1, nh=1, grid=(1, 256, 256), core=(1, 1, 1), halo=(0, 0, 0)), False),  # 65536 tiles
        (dict(B=1, nh=1, grid=(1, 255, 257), core=(1, 1, 1), halo=(0, 0, 0)), True),  # 65535 tiles
        (dict(B=256, nh=256, grid=(1, 8, 8), core=(1, 8, 8), halo=(0, 0, 0)), False),  # B * nh = 65536
        (dict(B=255, nh=257, grid=(1, 8, 8), core=(1, 8, 8), halo=(0, 0, 0)), True),  # B * nh = 65535
        (dict(B=1, nh=1, grid=(1, 1, 1), core=(1, 1, 1), halo=(0, 0, 0)), True),  # one token
    ],
)
def test_size_limits(lib, kw, ok):
    """Descriptors at the edges of the index ranges the kernels use (32-bit
    token and row indices, 16-bit tile and batch*head grid dimensions) are
    accepted up to the limit and refused beyond it, on the host."""
    d = _desc(**kw)
    assert (gattn.gattn_validate(d) == 0) == ok
    assert (gattn.gattn_saved_bytes(d) > 0) == ok


def test_fwd_rejects_bad_pointers_without_touching_the_gpu(lib):
    d = _desc()
    # NULL and misaligned pointers are refused before any CUDA call
    assert gattn.gattn_fwd(d, None, None, None, None, None, saved_bytes=0, stream=0) == 1
    assert gattn.gattn_fwd(d, 8, 16, 16, 16, 16, saved_bytes=1 << 40, stream=0) == 1
    # too-small saved buffer
    assert gattn.gattn_fwd(d, 16, 16, 16, 16, 16, saved_bytes=16, stream=0) == 3
    assert gattn.gattn_bwd(d, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, saved_bytes=1 << 40, ws_bytes=16, stream=0) == 3


def test_serve_request_bytes_on_host(lib):
    cfg = gattn.serve_cfg(d=64, Y=32, X=64, core=(1, 16, 16), halo=(0, 4, 4))
    T, nh = 4, 8
    b = gattn.gattn_serve_request_bytes(cfg, T, nh)
    N = T * 32 * 64
    assert b >= 2 * nh * N * 64 * 2  # state + attention output (BF16)
    assert gattn.gattn_serve_request_bytes(cfg, 0, nh) == 0
    assert gattn.gattn_serve_request_bytes(cfg, 2 * T, nh) > b


def test_serve_entry_points_refuse_null_on_the_host(lib):
    """The serving calls check their handle and pointers before any CUDA call."""
    assert gattn.gattn_serve_take_async(None, 1, None) == 1
    assert gattn.gattn_serve_copied(None, 1)[0] == 1
    assert gattn.gattn_serve_release(None, 1) == 1
    assert gattn.gattn_serve_poll(None, 1)[0] == 1


def test_compress_validation_on_the_host(lib):
    """Temporal-compression descriptors and pointers are checked before any launch."""
    d = gattn.gattn_compress_desc()
    d.B, d.nh, d.d, d.S, d.M, d.in_dtype, d.out_dtype = 1, 8, 128, 2048, 2048, gattn.GATTN_BF16, gattn.GATTN_BF16
    # 64 location blocks x 8 heads = 512 units < 152 x 16: the frames are split
    ws = gattn.gattn_compress_workspace_bytes(d)
    splits = ws // (8 * 2048 * (128 + 2) * 4)
    assert ws == splits * 8 * 2048 * 130 * 4 and splits >= 2
    d.M = 152 * 16 * 32  # enough location blocks: no split, no workspace
    assert gattn.gattn_compress_workspace_bytes(d) == 0
    for field, bad in (("S", 0), ("M", 0), ("d", 32), ("d", 96), ("B", 0)):
        e = gattn.gattn_compress_desc()
        e.B, e.nh, e.d, e.S, e.M, e.in_dtype, e.out_dtype = 1, 2, 64, 16, 16, gattn.GATTN_BF16, gattn.GATTN_FP32
        setattr(e, field, bad)
        assert gattn.gattn_compress_workspace_bytes(e) == 0
        assert gattn.gattn_compress_fwd(e, 16, 16, 16, 16, None, None, stream=0) == 1
    e.d = 64
    e.S = 16
    e.B = 1
    # null or misaligned pointers
    assert gattn.gattn_compress_fwd(e, None, 16, 16, 16, None, None, stream=0) == 1
    assert gattn.gattn_compress_fwd(e, 16, 24, 16, 16, None, None, stream=0) == 1


def test_gated_dps_linear_sizes_and_validation_on_the_host(lib):
    """Workspace queries and argument checks of the gated, posterior-sampling
    and linear-attention entry points, without a GPU."""
    d = _desc()
    saved = gattn.gattn_saved_bytes(d)
    nd = 2 * 3 * 4 * 16 * 32 * 64
    # gated: saved state (reused by both branches) + the cross branch's output
    assert gattn.gattn_gated_workspace_bytes(d) >= saved + nd * 2
    assert gattn.gattn_gated_fwd(d, None, 16, 16, 16, 16, 16, 16, 16, ws_bytes=1 << 30, stream=0) == 1
    # posterior sampling needs FP32 outputs (D and the gradients)
    assert gattn.gattn_dps_workspace_bytes(d) == 0
    d32 = _desc(out_dtype="fp32")
    need = gattn.gattn_dps_workspace_bytes(d32)
    assert need >= saved + gattn.gattn_bwd_workspace_bytes(d32) + 4 * nd * 4 + nd * 2
    p = gattn.gattn_dps_params()
    p.sigma, p.sigma_next, p.lam = 1.0, 0.5, 1.0
    assert gattn.gattn_dps_step(d32, p, None, 16, 16, 16, 16, 16, ws_bytes=need, stream=0) == 1
    p.sigma_next = 2.0  # noise must not grow
    assert gattn.gattn_dps_step(d32, p, 16, 16, 16, 16, 16, 16, ws_bytes=need, stream=0) == 1
    # linear attention: BF16, d = 64 only; workspace grows with the chunks
    ld = gattn.gattn_linear_desc()
    ld.B, ld.nh, ld.d, ld.N, ld.in_dtype, ld.out_dtype = 1, 2, 64, 4096, gattn.GATTN_BF16, gattn.GATTN_BF16
    small = gattn.gattn_linear_workspace_bytes(ld)
    assert small >= 2 * 64 * 64 * 4
    ld.N = 1 << 20
    assert gattn.gattn_linear_workspace_bytes(ld) > small
    ld.d = 128
    assert gattn.gattn_linear_workspace_bytes(ld) == 0
    assert gattn.gattn_linear_fwd(ld, 16, 16, 16, 16, 16, ws_bytes=1 << 30, stream=0) == 1
    ld.d, ld.N = 64, 0
    assert gattn.gattn_linear_fwd(ld, 16, 16, 16, 16, 16, ws_bytes=1 << 30, stream=0) == 1


def _extents(G, c, h):
    return [min((k + 1) * c + h, G) - max(k * c - h, 0) for k in range(-(-G // c))]


@pytest.mark.parametrize(
    "grid,core,halo",
    [((32, 64, 128), (32, 16, 32), (0, 4, 8)), ((32, 64, 128), (1, 16, 16), (0, 4, 4)),
     ((2048, 32, 64), (128, 32, 64), (8, 0, 0)), ((7, 32, 64), (1, 16, 16), (0, 4, 4)),
     ((3, 10, 13), (2, 4, 5), (1, 2, 2)), ((16, 256, 256), (16, 64, 64), (0, 8, 8))],
)
def test_block_shape_minimises_padded_work(lib, grid, core, halo):
    """The tensor-core kernels cut every extended tile into boxes of at most 128
    tokens, one 128-row MMA block each; the library's shape must minimise the
    padded work sum_tiles (number of boxes)^2 over every such shape."""
    d = gattn.make_desc(1, 1, 64, grid, core, halo, in_dtype="bf16")
    st, box = gattn.gattn_block_shape(d)
    assert st == 0 and all(b >= 1 for b in box) and box[0] * box[1] * box[2] <= 128
    ext = [_extents(grid[a], core[a], halo[a]) for a in range(3)]

    def cost(b):
        out = 1
        for a in range(3):
            out *= sum((-(-e // b[a])) ** 2 for e in ext[a])
        return out

    best = min(cost((bt, by, bx)) for bt in range(1, 129) for by in range(1, 128 // bt + 1)
               for bx in range(1, 128 // (bt * by) + 1))
    assert cost(box) == best


def test_block_shape_of_the_paper_and_small_tile_regimes(lib):
    # Tiles = 16 on 32 x 64 x 128: 4 x 4 x 8 boxes tile every extended tile exactly
    st, box = gattn.gattn_block_shape(gattn.make_desc(4, 16, 64, (32, 64, 128), (32, 16, 32), (0, 4, 8)))
    assert st == 0 and box == (4, 4, 8)
    # 16 x 16 cores with a 4-token halo: 24 x 24 extended tiles in five 5 x 24 boxes
    st, box = gattn.gattn_block_shape(gattn.make_desc(4, 16, 64, (32, 64, 128), (1, 16, 16), (0, 4, 4)))
    assert st == 0 and box == (1, 5, 24)
    assert gattn.gattn_block_shape(_desc(d=48))[0] == 1
