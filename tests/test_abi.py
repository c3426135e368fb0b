"""The C-ABI library builds, loads without a GPU and exports every symbol of include/hca.h."""

import ctypes
import os
import re

import pytest

from paper_2105_00448_gb300 import _build, hca

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return hca.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hca.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hca_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(hca.EXPORTS)


def test_config_struct_layout_matches(lib):
    cfg = hca.hca_config()
    assert lib.hca_config_default(ctypes.byref(cfg), 8, 9, 10) == 0
    assert cfg.struct_size == ctypes.sizeof(hca.hca_config)
    assert (cfg.nx, cfg.ny, cfg.nz) == (8, 9, 10)
    # Table 1 defaults arrive intact through the struct
    assert cfg.D_K == 1.05e5 and cfg.phi_K == 900.0 and cfg.K1 == 2.5 and cfg.K0 == 20.0
    assert cfg.r_K == 1.88e4 and list(cfg.D_G) == [9.6e3] * 3 and list(cfg.psi_G) == [1e-2] * 3
    assert cfg.T_cycle == 3.74 * 24 * 60 and cfg.K_phi == 1.4
    assert (cfg.k1, cfg.k1p, cfg.K_p53) == (4e-4, 0.01, 0.01)
    assert (cfg.k2, cfg.k2p, cfg.k2pp, cfg.J5, cfg.K_V) == (2e-3, 0.01, -2e-4, 0.04, 0.01)
    assert cfg.stream is None


def test_status_strings(lib):
    for code in range(0, -10, -1):
        s = lib.hca_status_string(code)
        assert s and s != b"unknown status"
    assert lib.hca_status_string(-99) == b"unknown status"


def test_argument_errors_without_gpu(lib):
    # calls that fail validation before touching the device
    assert lib.hca_config_default(None, 1, 1, 1) == hca.HCA_ERR_ARG
    bad = hca.make_config(4, 4, 4, n_drugs=5)
    h = ctypes.c_void_p()
    assert lib.hca_create(ctypes.byref(bad), None, None, None, 0, ctypes.byref(h)) == hca.HCA_ERR_ARG
    assert lib.hca_step(None, 1) == hca.HCA_ERR_ARG
    assert lib.hca_launch_count(None) == -1


def test_make_config_overrides(lib):
    cfg = hca.make_config(5, 6, 7, precision="f32", n_drugs=2, seed=2**40 + 3, kill_b=(2, 3, 1), dt=30.0)
    assert cfg.precision == hca.HCA_FP32 and cfg.n_drugs == 2 and cfg.seed == 2**40 + 3
    assert list(cfg.kill_b) == [2, 3, 1] and cfg.dt == 30.0
    with pytest.raises(KeyError):
        hca.make_config(5, 5, 5, no_such_field=1)


def test_library_defaults_equal_oracle_defaults(lib):
    """Every parameter the library and the oracle share has the same default
    (the GPU tests rely on this when they pass only overrides to both)."""
    from oracle import params as Pm

    cfg = hca.hca_config()
    assert lib.hca_config_default(ctypes.byref(cfg), 8, 9, 10) == 0
    ref = Pm.Config(8, 9, 10)
    skip = {"nx", "ny", "nz", "precision", "seed", "dose_peak"}
    shared = [f for f, _ in hca.hca_config._fields_ if f in Pm.Config.__dataclass_fields__ and f not in skip]
    assert len(shared) >= 40
    for f in shared:
        got, want = getattr(cfg, f), getattr(ref, f)
        got = list(got) if hasattr(got, "__len__") else got
        want = list(want) if isinstance(want, tuple) else want
        assert got == pytest.approx(want, rel=1e-15), f


def test_checkpoint_errors_without_gpu(lib, tmp_path):
    """hca_load rejects a missing file and a file that is not a checkpoint
    before touching the device; hca_save rejects null arguments."""
    h = ctypes.c_void_p()
    missing = str(tmp_path / "none.ckpt").encode()
    assert lib.hca_load(missing, None, ctypes.byref(h)) == hca.HCA_ERR_IO
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"NOTACKPT" + bytes(200))
    assert lib.hca_load(str(bad).encode(), None, ctypes.byref(h)) == hca.HCA_ERR_ARG
    assert lib.hca_load(None, None, ctypes.byref(h)) == hca.HCA_ERR_ARG
    assert lib.hca_save(None, b"x") == hca.HCA_ERR_ARG
    with pytest.raises(ValueError):
        hca.checkpoint_configs(str(bad))
