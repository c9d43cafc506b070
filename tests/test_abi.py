"""The C-ABI library builds, loads and exports every symbol the header declares; the ctypes
structures match the C layout; argument errors are reported without touching a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dirac.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1107_4650_gb300 import build as B
    B.build()
    import paper_1107_4650_gb300 as D
    return D.load_library()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(dirac_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ("dirac_create_grid", "dirac_set_potential", "dirac_step", "dirac_observables",
                 "dirac_set_state", "dirac_get_state", "dirac_destroy"):
        assert want in names


def test_binding_constants_match_the_header():
    """Every DIRAC_* enumerator of the header has the same value in the Python binding."""
    import paper_1107_4650_gb300 as D
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(DIRAC_[A-Z0-9_]+)\s*=\s*(-?\d+)\s*[,}\n]", text))
    assert "DIRAC_PLAN_3D_STRANG_ZPASS" in consts and len(consts) > 20
    wrong = {k: (v, getattr(D, k, None)) for k, v in consts.items() if getattr(D, k, None) != v}
    assert not wrong, wrong


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layout_matches_c(tmp_path):
    import paper_1107_4650_gb300 as D
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "dirac.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(dirac_config), sizeof(dirac_obs), sizeof(dirac_info),'
                   'offsetof(dirac_config, stream), offsetof(dirac_config, points_per_lane), offsetof(dirac_info, device_bytes),'
                   'offsetof(dirac_config, ext_state), offsetof(dirac_info, state_index));'
                   'return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(D.dirac_config), ctypes.sizeof(D.dirac_obs), ctypes.sizeof(D.dirac_info),
                    D.dirac_config.stream.offset, D.dirac_config.points_per_lane.offset,
                    D.dirac_info.device_bytes.offset, D.dirac_config.ext_state.offset, D.dirac_info.state_index.offset]


def test_ext_state_needs_both_buffers(lib):
    """One caller-owned ping-pong buffer without the other is an argument error, reported before any CUDA call."""
    import paper_1107_4650_gb300 as D
    for pair in ((4096, None), (None, 4096)):
        cfg = D.make_config((64, 1, 64))
        cfg.ext_state[0], cfg.ext_state[1] = pair
        with pytest.raises(D.DiracError) as e:
            D.dirac_create_grid(cfg)
        assert e.value.status == D.DIRAC_ERR_ARG and "ext_state" in D.dirac_last_error(None)


def test_version_and_defaults(lib):
    import paper_1107_4650_gb300 as D
    assert "sm_103a" in D.dirac_version()
    cfg = D.dirac_default_config()
    assert cfg.ndim == 2 and cfg.n[1] == 1 and abs(cfg.c - 137.0359895) < 1e-12 and cfg.flux_face == -1


@pytest.mark.parametrize("field,value", [("ndim", 4), ("precision", 7), ("boundary", 5), ("flux_face", 0),
                                         ("steps_per_launch", 3), ("points_per_lane", 3), ("dx", -1.0)])
def test_invalid_config_is_rejected_before_any_cuda_call(lib, field, value):
    import paper_1107_4650_gb300 as D
    cfg = D.make_config((64, 1, 64))
    setattr(cfg, field, value)
    with pytest.raises(D.DiracError) as e:
        D.dirac_create_grid(cfg)
    assert e.value.status == D.DIRAC_ERR_ARG
    assert D.dirac_last_error(None)


def test_2d_grid_needs_ny_1(lib):
    import paper_1107_4650_gb300 as D
    cfg = D.make_config((64, 2, 64))
    with pytest.raises(D.DiracError) as e:
        D.dirac_create_grid(cfg)
    assert e.value.status == D.DIRAC_ERR_ARG


def test_injected_allocation_failure(lib, monkeypatch):
    import paper_1107_4650_gb300 as D
    monkeypatch.setenv("DIRAC_INJECT_OOM", "1")
    with pytest.raises(D.DiracError) as e:
        D.dirac_create_grid(D.make_config((64, 1, 64)))
    assert e.value.status == D.DIRAC_ERR_OOM


def test_null_handles_are_errors_not_crashes(lib):
    import paper_1107_4650_gb300 as D
    assert lib.dirac_step(None, 1) == D.DIRAC_ERR_ARG
    assert lib.dirac_destroy(None) == D.DIRAC_OK
    assert lib.dirac_set_state(None, None, 0) == D.DIRAC_ERR_ARG


def test_batch_rejects_bad_runs_without_a_gpu(lib):
    import paper_1107_4650_gb300 as D
    cfg = D.dirac_batch_default_config()
    bad = [{"side": 64, "face": 64, "nsteps": 10, "V0": 1.0, "L": 0.01, "p0": 1.0, "width": 0.01, "x0": -0.05}]
    with pytest.raises(D.DiracError) as e:
        D.dirac_batch_create(bad, cfg)
    assert e.value.status == D.DIRAC_ERR_ARG
    cfg.precision = 5
    ok = [dict(bad[0], face=32)]
    with pytest.raises(D.DiracError) as e:
        D.dirac_batch_create(ok, cfg)
    assert e.value.status == D.DIRAC_ERR_ARG


def test_strang_3d_runs_one_step_per_block(lib):
    import paper_1107_4650_gb300 as D
    cfg = D.make_config((16, 16, 16), ndim=3, splitting=D.DIRAC_STRANG, steps_per_launch=2)
    with pytest.raises(D.DiracError) as e:
        D.dirac_create_grid(cfg)
    assert e.value.status == D.DIRAC_ERR_ARG


def test_3d_steps_per_launch_validation(lib):
    """3-D grids run one or two steps per launch, two only in the fused pass (points_per_lane 0)."""
    import paper_1107_4650_gb300 as D
    for kw in (dict(steps_per_launch=4), dict(steps_per_launch=2, points_per_lane=2),
               dict(steps_per_launch=2, points_per_lane=1)):
        cfg = D.make_config((16, 16, 16), ndim=3, **kw)
        with pytest.raises(D.DiracError) as e:
            D.dirac_create_grid(cfg)
        assert e.value.status == D.DIRAC_ERR_ARG


def test_fx64_validation(lib):
    """DIRAC_FX64 runs first-order steps (one or, in 2-D, two per launch) and second-order steps (one per launch
    block; 3-D as single sweeps, single sweeps with a z-phase-z pass, or fused passes)."""
    import paper_1107_4650_gb300 as D
    for n, kw in (((8, 8, 8), dict(ndim=3, steps_per_launch=2)), ((8, 8, 8), dict(ndim=3, splitting=D.DIRAC_STRANG,
                                                                                     steps_per_launch=2)),
                  ((16, 1, 16), dict(splitting=D.DIRAC_STRANG, steps_per_launch=2)),
                  ((16, 1, 16), dict(splitting=D.DIRAC_STRANG, steps_per_launch=1, points_per_lane=4)),
                  ((16, 1, 16), dict(char_shift=2)), ((16, 1, 16), dict(steps_per_launch=4)),
                  ((16, 1, 16), dict(steps_per_launch=2, points_per_lane=4)), ((16, 1, 16), dict(precision=3))):
        kw.setdefault("precision", D.DIRAC_FX64)
        cfg = D.make_config(n, **kw)
        with pytest.raises(D.DiracError) as e:
            D.dirac_create_grid(cfg)
        assert e.value.status == D.DIRAC_ERR_ARG


def test_char_shift_validation(lib):
    import paper_1107_4650_gb300 as D
    for kw in (dict(char_shift=5), dict(char_shift=-1), dict(char_shift=2, ndim=3, n=(8, 8, 8), points_per_lane=2),
               dict(char_shift=2, splitting=D.DIRAC_STRANG, points_per_lane=2), dict(char_shift=3, steps_per_launch=2),
               dict(char_shift=2, points_per_lane=4), dict(char_shift=2, precision=D.DIRAC_FX64),
               dict(char_shift=3, boundary=D.DIRAC_BC_PERIODIC, flux_face=2),
               dict(char_shift=2, boundary=D.DIRAC_BC_PERIODIC, flux_face=15),
               dict(char_shift=4, boundary=D.DIRAC_BC_PERIODIC, flux_face=3, ndim=3, n=(8, 8, 8))):
        n = kw.pop("n", (16, 1, 16))
        cfg = D.make_config(n, **kw)
        with pytest.raises(D.DiracError) as e:
            D.dirac_create_grid(cfg)
        assert e.value.status == D.DIRAC_ERR_ARG
