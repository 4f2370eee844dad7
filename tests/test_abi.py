"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/gsr.h declares, agrees with
the ctypes binding on struct layouts, and rejects bad arguments before it
touches the device."""
import ctypes
import subprocess

import pytest

from paper_2411_17660_b300 import binding as B
from paper_2411_17660_b300 import build as Build


@pytest.fixture(scope="module")
def lib():
    Build.build()
    return B.load()


def test_exports_every_declared_function(lib):
    declared = B.declared_functions()
    assert len(declared) >= 11
    out = subprocess.run(["nm", "-D", "--defined-only", Build.LIB], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    for f in declared:
        getattr(lib, f)


def test_struct_layouts_match_binding(lib):
    for i, s in enumerate(B.ABI_STRUCTS):
        assert lib.gsr_abi_sizeof(i) == ctypes.sizeof(s), s.__name__
    assert lib.gsr_abi_sizeof(99) == 0
    assert lib.gsr_abi_version() == B.ABI_VERSION


def test_status_strings(lib):
    for code, name in B.STATUS.items():
        assert lib.gsr_status_string(code).decode() == name


def test_create_rejects_bad_config(lib):
    for tile in (8, 16, 32):
        B.Context(tile)
    for tile in (4, 12, 64):
        with pytest.raises(B.GsrError):
            B.Context(tile)
    with pytest.raises(B.GsrError):
        B.Context(16, flags=4)
    # the forward blend's block height: 8 everywhere, 16 at tiles 16 and 32 (0: the default)
    for tile, rows in ((8, 8), (16, 8), (16, 16), (32, 8), (32, 16), (8, 0), (16, 0)):
        B.Context(tile, fwd_rows=rows)
    for tile, rows in ((8, 16), (16, 4), (16, 12), (32, 32)):
        with pytest.raises(B.GsrError):
            B.Context(tile, fwd_rows=rows)


def _view(H=32, W=48):
    return B.View(H, W, 40.0, 40.0, W / 2, H / 2, 0x1000, 0x2000, 0, 0)


def test_workspace_size_is_monotone(lib):
    c = B.Context(16)
    a = c.workspace_size(1000, [_view()], 1 << 20)
    b = c.workspace_size(1000, [_view()], 1 << 21)
    d = c.workspace_size(2000, [_view(), _view(64, 64)], 1 << 20)
    assert 0 < a < b and a < d
    assert b - a >= 24 * (1 << 20)  # two key/value buffers per key


def test_argument_errors_return_einval_without_device(lib):
    c = B.Context(16)
    g = B.Gaussians(10, 0, 0x100, 0x100, 0x100, 0x100, 0x100)
    # V = 0
    assert c.render(g, [], 0x1000, 1 << 20, 0) == B.EINVAL
    # bad intrinsics
    bad = _view()
    bad.fx = -1.0
    assert c.render(g, [bad], 0x1000, 1 << 20, 0) == B.EINVAL
    # unaligned workspace
    assert c.render(g, [_view()], 0x1001, 1 << 30, 0) == B.EINVAL
    # workspace too small for any key
    assert c.render(g, [_view()], 0x1000, 4096, 0) == B.EINVAL
    # SH degree out of range
    g4 = B.Gaussians(10, 4, 0x100, 0x100, 0x100, 0x100, 0x100)
    assert c.render(g4, [_view()], 0x1000, 1 << 30, 0) == B.EINVAL
    # null parameter pointer
    g0 = B.Gaussians(10, 0, 0, 0x100, 0x100, 0x100, 0x100)
    assert c.render(g0, [_view()], 0x1000, 1 << 30, 0) == B.EINVAL
    assert "NULL" in lib.gsr_last_error(c.h).decode()
    # backward without a forward on that workspace
    out = B.Grads(0x100, 0x100, 0x100, 0x100, 0x100, 0, 0, 0, 0)
    vg = [B.ViewGrad(0, 0, 0, 0)]
    assert c.render_backward(g, [_view()], vg, out, 0x1000, 1 << 30, 0) == B.ENOTREADY
