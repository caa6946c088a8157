"""MD checkpoint files on the host: a save/load round trip returns the arrays
bit for bit and the scalars exactly; a file of another format is refused.
CPU only (the module is loaded by path: it needs no GPU library)."""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ck():
    spec = importlib.util.spec_from_file_location(
        "tb_checkpoint", os.path.join(ROOT, "paper_0910_4497_gb300", "checkpoint.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_round_trip(tmp_path):
    m = ck()
    rng = np.random.default_rng(3)
    pos, vel, F = (rng.standard_normal((17, 3)) for _ in range(3))
    path = tmp_path / "state.npz"
    m.save(path, pos, vel, F, 25.0, 123, 1004, params={"r": 16, "Rc": 6.5}, prec="mixed")
    st = m.load(path)
    for k, a in (("pos", pos), ("vel", vel), ("F", F)):
        assert np.array_equal(st[k], a)
    assert st["L"] == 25.0 and st["step"] == 123 and st["seed"] == 1004
    assert st["params"] == {"r": 16, "Rc": 6.5} and st["prec"] == "mixed"


def test_refuses_other_format_and_bad_shapes(tmp_path):
    m = ck()
    z = np.zeros((2, 3))
    with pytest.raises(ValueError):
        m.save(tmp_path / "bad.npz", z, np.zeros((3, 3)), z, 1.0, 0, 0)
    path = tmp_path / "old.npz"
    np.savez(path, format=np.int64(m.FORMAT + 1), pos=z, vel=z, F=z, L=1.0, step=0, seed=0,
             params=np.array("{}"), prec=np.array(""))
    with pytest.raises(ValueError):
        m.load(path)
