"""Host-side checks of the C ABI (no GPU needed): the library builds and loads, exports every
function include/dscf.h declares, and validates parameters before touching a device."""
import ctypes
import os
import re

import pytest

from paper_1204_2088_gb300 import build, dscf, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dscf.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "sizeof")))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "dscf_init" in names and "lb_step" in names and "dscf_densities" in names
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_bytes_validates_parameters(lib):
    cfg = inputs.melt((16, 12, 10), 8, 0.5, 10.0)
    ok = dscf.workspace_bytes(cfg, dscf.FP64)
    assert ok > 0
    assert dscf.workspace_bytes(cfg, dscf.FP32) < ok
    for bad in [dict(N=1), dict(nA=0), dict(nA=8), dict(tau_s=0.5), dict(cn_sweeps=3), dict(ncg_iters=40),
                dict(a=2.0), dict(grid=(0, 4, 4)), dict(phi_p=0.5)]:
        c = dict(cfg)
        c.update(bad)
        assert dscf.workspace_bytes(c, dscf.FP64) == 0, bad
    c = dict(cfg); c["chi"] = {(0, 0): 0.1}
    assert dscf.workspace_bytes(c, dscf.FP64) == 0
    # mixed replicas must share the step structure
    c2 = dict(cfg); c2["ncg_iters"] = 2
    assert dscf.workspace_bytes([cfg, c2], dscf.FP64) == 0
    assert dscf.workspace_bytes([cfg, inputs.melt((8, 8, 8), 6, 0.5, 10.0)], dscf.FP64) > ok
    assert dscf.workspace_bytes(cfg, 7) == 0


def test_workspace_scales_with_chain_and_grid(lib):
    a = dscf.workspace_bytes(inputs.melt((32, 32, 32), 16, 0.5, 10.0), dscf.FP32)
    b = dscf.workspace_bytes(inputs.melt((32, 32, 32), 32, 0.5, 10.0), dscf.FP32)
    c = dscf.workspace_bytes(inputs.melt((64, 32, 32), 16, 0.5, 10.0), dscf.FP32)
    z = dscf.workspace_bytes(inputs.melt((8, 8, 8), 16, 0.5, 10.0), dscf.FP32)   # fixed parts + 512 sites
    assert b - a >= 16 * 32 ** 3 * 4          # 16 more propagator slices
    assert c - a > 0.9 * (a - z)              # twice the sites: about twice the per-site part


def test_net_workspace_validates_and_holds_the_padded_tcgen05_copies(lib):
    """The network workspace: 0 for grids it cannot run (nx not a multiple of 16, empty extents,
    no samples); on a grid the tcgen05 forward takes (nx a multiple of 128, ny of 8) it also
    holds the padded channel-group copies of the layer inputs, rows x (nx + 4) sites of 16 (x16f)
    and 32 (h1p, h2p) BF16 channels, and nothing else beyond a grid of as many sites that the
    tcgen05 path does not take."""
    f = lib.dscf_net_workspace_bytes
    for bad in [(8, 8, 8, 1), (24, 8, 8, 1), (128, 0, 4, 1), (128, 8, 0, 1), (128, 8, 4, 0)]:
        assert f(*bad) == 0, bad
    for nx, ny, nz, B in [(128, 8, 4, 1), (128, 16, 8, 2), (256, 8, 4, 1)]:
        rows = ny * nz * B
        padded = rows * (nx + 4) * (16 + 32 + 32) * 2
        other = f(16, ny * nx // 16, nz, B)     # same sites, rows of 16: mma.sync only
        assert f(nx, ny, nz, B) - other == padded, (nx, ny, nz, B)


def test_init_rejects_null_output(lib):
    p = dscf.make_params(inputs.melt((8, 8, 8), 4, 0.5, 10.0))
    rc = lib.dscf_init(ctypes.byref(p), 1, 0, None, 0, None, None)
    assert rc == -1
    assert b"NULL" in lib.dscf_last_error(None)


def test_init_tuned_rejects_null_output(lib):
    p = dscf.make_params(inputs.melt((8, 8, 8), 4, 0.5, 10.0))
    rc = lib.dscf_init_tuned(ctypes.byref(p), 1, 0, None, 0, None, 4, 1, None)
    assert rc == -1


def test_tuning_cache_round_trip(tmp_path):
    path = str(tmp_path / "tuning.json")
    assert dscf._tuning_cache_read(path) == {}
    dscf._tuning_cache_write(path, "a", (16, 0))
    dscf._tuning_cache_write(path, "b", (8, 4))
    dscf._tuning_cache_write(path, "a", (11, 2))
    assert dscf._tuning_cache_read(path) == {"a": (11, 2), "b": (8, 4)}
    with open(path, "w") as f:
        f.write("{not json")
    assert dscf._tuning_cache_read(path) == {}


def test_binding_names_every_declared_error_code():
    """The status codes of include/dscf.h and the binding's table of names agree."""
    text = open(os.path.join(ROOT, "include", "dscf.h")).read()
    codes = {int(v): n for n, v in re.findall(r"\b(DSCF_ERR_\w+)\s*=\s*(-\d+)", text)}
    assert codes and codes == dscf.ERRORS
