"""The oracle's and the library's default parameters against Table 1 of the
paper, transcribed in tests/golden/table1_parameters.txt."""

import ctypes
import os

import pytest

from oracle import params as Pm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_parameters.txt")


def table1():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        name, value = line.split()[:2]
        out[name] = [float(v) for v in value.split(",")]
    return out


def test_oracle_defaults_are_table1():
    cfg = Pm.Config(4, 4, 4)
    t = table1()
    assert len(t) >= 25
    for name, vals in t.items():
        if name == "plasma_decay_0":
            got = [cfg.plasma_decay[0]]
        else:
            got = getattr(cfg, name)
            got = list(got) if isinstance(got, tuple) else [got]
        if len(vals) == 1 and len(got) > 1:
            vals = vals * len(got)
        assert got == pytest.approx(vals, rel=1e-9), name


def test_library_defaults_are_table1():
    from paper_2105_00448_gb300 import hca

    lib = hca.load()
    cfg = hca.hca_config()
    assert lib.hca_config_default(ctypes.byref(cfg), 4, 4, 4) == 0
    for name, vals in table1().items():
        if name == "plasma_decay_0":
            got = [cfg.plasma_decay[0]]
        else:
            got = getattr(cfg, name)
            got = list(got) if hasattr(got, "__len__") else [got]
        if len(vals) == 1 and len(got) > 1:
            vals = vals * len(got)
        assert got == pytest.approx(vals, rel=1e-9), name
