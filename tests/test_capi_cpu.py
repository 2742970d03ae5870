"""C ABI checks that need no GPU: the library builds, loads, exports every declared symbol,
and rejects invalid arguments before touching the device."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2206_13164_gb300 import nrmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    inc = os.path.join(ROOT, "include")
    for h in os.listdir(inc):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            syms |= set(re.findall(r"\b(nrmg_[a-z_0-9]+)\s*\(", src))
    return sorted(syms)


def test_library_exports_every_declared_symbol():
    path = nrmg.lib()._name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    assert len(declared_symbols()) >= 21


def test_library_is_built_for_sm103a():
    out = subprocess.run(["cuobjdump", "--list-elf", nrmg.lib()._name], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def _args(nx=32, ny=32, levels=3, M=5, order=1, slope=0, precision=0):
    return (nrmg.Grid(nx, ny, 1.0, 1.0, levels), M, nrmg.Opts(order, slope, 0.9, 2, 2, 4, 1, precision, 0.0))


def test_workspace_bytes_and_argument_checks():
    L = nrmg.lib()
    g, M, o = _args()
    n = L.nrmg_workspace_bytes(ctypes.byref(g), M, ctypes.byref(o))
    assert n > 0
    # grows with the grid and with M
    g2, _, _ = _args(nx=64, ny=64, levels=4)
    assert L.nrmg_workspace_bytes(ctypes.byref(g2), M, ctypes.byref(o)) > 3 * n
    assert L.nrmg_workspace_bytes(ctypes.byref(g), 8, ctypes.byref(o)) > n
    bad = [
        _args(nx=30, levels=3),      # not divisible by 2^(levels-1)
        _args(levels=0),
        _args(M=2),                  # M >= 3 required
        _args(order=3),
        _args(slope=5),
        _args(precision=2),          # 0 FP64, 1 mixed
    ]
    for g, M, o in bad:
        assert L.nrmg_workspace_bytes(ctypes.byref(g), M, ctypes.byref(o)) == 0


def test_create_rejects_invalid_arguments_without_a_device():
    L = nrmg.lib()
    g, M, o = _args()
    walls = (nrmg.Wall * 4)()
    for w in walls:
        w.theta, w.chi = 1.0, 1.0
    coll = nrmg.Collision(0, 2 / 3, 0.81, 1.0)
    ctx = ctypes.c_void_p()
    ws = ctypes.c_void_p(256)  # never dereferenced: every case below fails its argument check
    # Kn <= 0
    assert L.nrmg_create(ctypes.byref(g), M, 0.0, walls, ctypes.byref(coll), ctypes.byref(o), ws, 1 << 40, None,
                         ctypes.byref(ctx)) == nrmg.ERR_ARG
    # a wall moving along its own normal (bottom wall, u_y != 0)
    walls[0].u = (ctypes.c_double * 3)(0.0, 0.1, 0.0)
    assert L.nrmg_create(ctypes.byref(g), M, 0.1, walls, ctypes.byref(coll), ctypes.byref(o), ws, 1 << 40, None,
                         ctypes.byref(ctx)) == nrmg.ERR_ARG
    walls[0].u = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    walls[2].theta = -1.0
    assert L.nrmg_create(ctypes.byref(g), M, 0.1, walls, ctypes.byref(coll), ctypes.byref(o), ws, 1 << 40, None,
                         ctypes.byref(ctx)) == nrmg.ERR_ARG
    walls[2].theta = 1.0
    # an unknown collision model (0 BGK, 1 Shakhov, 2 ES-BGK are the known ones)
    bad_coll = nrmg.Collision(3, 2 / 3, 0.81, 1.0)
    assert L.nrmg_create(ctypes.byref(g), M, 0.1, walls, ctypes.byref(bad_coll), ctypes.byref(o), ws, 1 << 40, None,
                         ctypes.byref(ctx)) == nrmg.ERR_ARG
    # workspace too small
    assert L.nrmg_create(ctypes.byref(g), M, 0.1, walls, ctypes.byref(coll), ctypes.byref(o), ws, 1024, None,
                         ctypes.byref(ctx)) == nrmg.ERR_OOM
    # misaligned workspace
    assert L.nrmg_create(ctypes.byref(g), M, 0.1, walls, ctypes.byref(coll), ctypes.byref(o), ctypes.c_void_p(264),
                         1 << 40, None, ctypes.byref(ctx)) == nrmg.ERR_ARG
    assert not ctx.value


def test_status_strings():
    L = nrmg.lib()
    assert L.nrmg_status_str(0) == b"NRMG_OK"
    assert L.nrmg_status_str(6) == b"NRMG_ERR_TIMEOUT"
    assert L.nrmg_last_error(None) == b""


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2206_13164_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                for bad in ("import oracle", "from oracle", "liboracle", "nrmg_oracle"):
                    assert bad not in txt, (f, bad)


def test_no_cpu_fallback_without_cuda(monkeypatch):
    import torch

    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    with pytest.raises(RuntimeError):
        nrmg.Solver(8, 8, 3, 0.1, [((0, 0, 0), 1.0, 1.0)] * 4)


def test_net_and_learned_entry_points_check_arguments():
    """Argument checks of the learned guess's C ABI, without touching a GPU."""
    import ctypes
    from ctypes import c_double, c_int, c_longlong, c_size_t, c_void_p

    L = nrmg.lib()
    L.nrmg_net_workspace_bytes.restype = c_size_t
    L.nrmg_net_workspace_bytes.argtypes = [c_int, c_int, c_int, c_longlong]
    assert L.nrmg_net_workspace_bytes(19, 64, 10, 4096) > 0
    assert L.nrmg_net_workspace_bytes(19, 32, 10, 4096) < L.nrmg_net_workspace_bytes(19, 64, 10, 4096)
    for bad in ((0, 64, 10, 4096), (65, 64, 10, 4096), (19, 48, 10, 4096), (19, 64, 17, 4096), (19, 64, 10, 0)):
        assert L.nrmg_net_workspace_bytes(*bad) == 0, bad
    L.nrmg_net_create.restype = c_int
    L.nrmg_net_create.argtypes = [c_int, c_int, c_int, c_longlong, ctypes.c_ulonglong, c_void_p, c_size_t, c_void_p,
                                  ctypes.POINTER(c_void_p)]
    h = c_void_p()
    assert L.nrmg_net_create(19, 64, 10, 4096, 0, None, 1 << 30, None, ctypes.byref(h)) == nrmg.ERR_ARG
    L.nrmg_net_param_count.restype = c_longlong
    L.nrmg_net_param_count.argtypes = [c_void_p]
    assert L.nrmg_net_param_count(None) == 0
    L.nrmg_learned_features.restype = c_int
    L.nrmg_learned_features.argtypes = [c_void_p, c_int, c_int, c_double, c_double, c_double, c_double, c_void_p,
                                        c_void_p, c_void_p]
    assert L.nrmg_learned_features(None, 4, 4, 1.0, 1.0, 0.1, 0.2, None, None, None) == nrmg.ERR_ARG
    L.nrmg_set_reference.restype = c_int
    L.nrmg_set_reference.argtypes = [c_void_p, c_double, c_double]
    assert L.nrmg_set_reference(None, 1.0, 1.0) == nrmg.ERR_ARG
    L.nrmg_set_state_from_fields.restype = c_int
    L.nrmg_set_state_from_fields.argtypes = [c_void_p, c_void_p]
    assert L.nrmg_set_state_from_fields(None, None) == nrmg.ERR_ARG
    assert L.nrmg_mixed_fallback(None) == 0


def test_noalloc_binding_checks_shapes_before_the_library():
    """residual_noalloc hands the library bare pointers: arrays of the wrong shape or on
    different devices are refused on the host."""
    import torch

    from inputs import lid_cavity

    prob = lid_cavity(16, 5, 0.1, 0.2)
    for P, F in ((torch.zeros(4, 4, dtype=torch.float64), torch.zeros(256, 56, dtype=torch.float64)),
                 (torch.zeros(256, 4, dtype=torch.float64), torch.zeros(256, 55, dtype=torch.float64)),
                 (torch.zeros(256, 4, dtype=torch.float64), torch.zeros(256, 56, dtype=torch.float64))):
        with pytest.raises(ValueError):
            nrmg.residual_noalloc(prob, P, F)


def test_autotune_cache_round_trip(tmp_path):
    """The sweep-grid cache: a stored result is found again under the same key (problem
    shapes sorted, scheme and model in the key), and writes replace the file atomically."""
    path = str(tmp_path / "tune.json")

    class O:
        order, slope, precision = 2, 2, 0

    key = "GB300/152sm|" + ";".join(sorted(["64x64:M5:L4", "128x128:M8:L5"])) + "|order2:slope2:prec0|model0"
    nrmg._tune_store(path, key, 2, {1: 0.5, 2: 0.4})
    nrmg._tune_store(path, key + "x", 3, {3: 0.1})
    data = nrmg._tune_load(path)
    assert data[key]["ctas_per_sm"] == 2 and data[key]["s_per_cycle"] == {"1": 0.5, "2": 0.4}
    assert data[key + "x"]["ctas_per_sm"] == 3
    assert nrmg._tune_load(str(tmp_path / "missing.json")) == {}
