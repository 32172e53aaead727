"""The C-ABI library loads and exports every entry point include/pic.h
declares; host-side configuration checks (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_1310_5284_gb300 import build
    build()
    from paper_1310_5284_gb300 import _abi
    return _abi


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(abi):
    names = declared_functions()
    assert len(names) >= 19
    lib = ctypes.CDLL(abi.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    # the binding declares exactly the header's entry points
    assert set(abi.SIGNATURES) == set(names)


def test_version_and_build_info(abi):
    assert abi.lib().pic_version() == 3
    assert b"sm_103a" in abi.lib().pic_build_info()


def _sizes(abi, cfg):
    from paper_1310_5284_gb300.sim import make_config
    c = make_config(cfg)
    s = abi.PicSizes()
    code = abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s))
    return code, s


def test_required_sizes_scale_with_capacity(abi):
    code, s1 = _sizes(abi, dict(workloads.CFG_SMALL_CCP))
    assert code == 0 and s1.arena_bytes > 0 and s1.snapshot_bytes > s1.arena_bytes
    code, s2 = _sizes(abi, dict(workloads.CFG_SMALL_CCP, capacity=100_000))
    assert code == 0
    # two buffers x two species x six 4-byte fields per extra slot
    extra = s2.arena_bytes - s1.arena_bytes
    assert extra >= 2 * 6 * 4 * (100_000 - 25_600)


def test_strict_mode_rejects_unstable_leapfrog(abi):
    # Eq. (1): omega_p dt < 2.  At n0 = 1.03e17 and dt = 1/(400 f), omega_p dt = 3.3
    cfg = dict(workloads.CFG_WIDE_EXPLICIT, dt=1.0 / (400 * 13.56e6), strict=True)
    code, _ = _sizes(abi, cfg)
    assert code == -2
    assert b"Eq. (1)" in abi.lib().pic_last_error(None)
    cfg["strict"] = False
    assert _sizes(abi, cfg)[0] == 0
    # the implicit schemes are exempt
    assert _sizes(abi, dict(cfg, scheme="ec_implicit", strict=True))[0] == 0
    assert _sizes(abi, dict(cfg, scheme="mc_implicit", strict=True))[0] == 0


def test_unknown_scheme_is_rejected(abi):
    from paper_1310_5284_gb300.sim import make_config
    c = make_config(dict(workloads.CFG_SMALL_CCP))
    s = abi.PicSizes()
    for scheme, code in ((0, 0), (1, 0), (2, 0), (3, 0), (4, 0), (5, -1), (-1, -1)):
        c.scheme = scheme
        assert abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s)) == code, scheme


def test_m3_scheme_limits(abi):
    """The m = 3 scheme: capacity below 2^23 a species (int64 headroom of
    charges of 6 * 2^36 a particle); single runs only."""
    from paper_1310_5284_gb300.sim import make_config
    c = make_config(dict(workloads.CFG_SMALL_CCP, scheme="ec3_explicit"))
    s = abi.PicSizes()
    assert abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s)) == 0
    c.capacity[0] = (1 << 23) - 1
    assert abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s)) == 0
    c.capacity[0] = 1 << 23
    assert abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s)) == -4
    arr = (abi.PicConfig * 2)(make_config(dict(workloads.CFG_SMALL_CCP)),
                              make_config(dict(workloads.CFG_SMALL_CCP, scheme="ec3_explicit")))
    assert abi.lib().pic_batch_required_sizes(arr, 2, ctypes.byref(s)) == -1
    assert b"m = 3" in abi.lib().pic_last_error(None)
    assert abi.lib().pic_batch_required_sizes(arr, 1, ctypes.byref(s)) == 0


@pytest.mark.parametrize("bad,code", [
    (dict(n_cells=1), -1), (dict(n_cells=2048), -1), (dict(capacity=1 << 29), -4),
    (dict(np_init=0), -1), (dict(dt=0.0), -1), (dict(eedf_bins=0), -1),
    (dict(ions_mobile=False), -1),  # collisions need mobile ions
])
def test_invalid_configs_are_rejected(abi, bad, code):
    cfg = dict(workloads.CFG_SMALL_CCP)
    cfg.update(bad)
    assert _sizes(abi, cfg)[0] == code


def test_init_rejects_small_or_misaligned_arena(abi):
    from paper_1310_5284_gb300.sim import make_config
    c = make_config(dict(workloads.CFG_SMALL_CCP))
    s = abi.PicSizes()
    abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s))
    h = ctypes.c_void_p()
    small = abi.PicBuffers(256, s.arena_bytes - 1)
    assert abi.lib().pic_init(ctypes.byref(c), ctypes.byref(small), None, ctypes.byref(h)) == -3
    odd = abi.PicBuffers(256 + 8, s.arena_bytes)
    assert abi.lib().pic_init(ctypes.byref(c), ctypes.byref(odd), None, ctypes.byref(h)) == -3
    assert not h.value


def test_wait_selftest_rejects_bad_arguments_before_any_launch(abi):
    st, waited = ctypes.c_uint32(), ctypes.c_double()
    assert abi.lib().pic_selftest_wait(-1, ctypes.byref(st), ctypes.byref(waited), None) == -1
    assert abi.lib().pic_selftest_wait(11 * 10 ** 9, ctypes.byref(st), ctypes.byref(waited), None) == -1
    assert abi.lib().pic_selftest_wait(1000, None, ctypes.byref(waited), None) == -1
    assert b"pic_selftest_wait" in abi.lib().pic_last_error(None)


def test_set_state_rejects_null_arguments_before_any_device_work(abi):
    hp = abi.PicHostParticles()
    assert abi.lib().pic_set_state(None, ctypes.byref(hp), ctypes.byref(hp)) == -1
    assert abi.lib().pic_set_particles(None, 0, ctypes.byref(hp)) == -1


def test_non_uniform_grid_configs(abi):
    """cell_width: positive widths summing to the gap, the EC schemes
    (explicit with m = 2 or 3, direct implicit) with mobile ions, single runs;
    the arena grows by the grid's tables."""
    from paper_1310_5284_gb300.sim import make_config
    base = dict(workloads.CFG_SMALL_CCP)
    s = abi.PicSizes()
    c = make_config(base)
    assert abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s)) == 0
    uniform = s.arena_bytes
    good = workloads.with_stretch(base, 0.6)
    c = make_config(good)
    assert abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s)) == 0
    assert s.arena_bytes > uniform
    n, length = base["n_cells"], base["length"]
    for bad in ([length / n] * (n - 1) + [0.0],                      # an empty cell
                [length / n] * (n - 1) + [-length / n],              # a negative width
                [1.01 * length / n] * n,                              # widths do not sum to the gap
                [length / n] * (n - 1) + [float("nan")]):
        c = make_config(dict(base, cell_width=bad))
        assert abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s)) == -1
    for scheme in ("ec_implicit", "ec3_explicit"):
        c = make_config(dict(good, scheme=scheme))
        assert abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s)) == 0, scheme
    for over in (dict(scheme="mc_explicit"), dict(scheme="mc_implicit"),
                 dict(ions_mobile=False, mcc=False, bg_density=1e15)):
        c = make_config(dict(good, **over))
        assert abi.lib().pic_required_sizes(ctypes.byref(c), ctypes.byref(s)) == -1, over
    arr = (abi.PicConfig * 1)(make_config(good))
    assert abi.lib().pic_batch_required_sizes(arr, 1, ctypes.byref(s)) == -1
