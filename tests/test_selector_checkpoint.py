"""Selector training checkpoints (host side, no GPU): the saved state
(parameters, Adam moments and step, the shuffling generator, the loss
history) comes back bit for bit, a restored generator continues the same
permutation sequence as one that was never interrupted, an interrupted
write leaves the previous checkpoint intact, and a file of another format
version or network size is refused."""
import json
import os

import numpy as np
import pytest

from paper_2606_25453_gb300 import SEL_NPARAM
from paper_2606_25453_gb300 import selector as sel


def state(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.standard_normal(SEL_NPARAM).astype(np.float32), rng.standard_normal(SEL_NPARAM).astype(np.float32),
            rng.random(SEL_NPARAM).astype(np.float32))


def test_round_trip_and_rng_continuation(tmp_path):
    path = str(tmp_path / "sel.ckpt")
    prm, m, v = state(1)
    rng = np.random.Generator(np.random.PCG64(5))
    ref = np.random.Generator(np.random.PCG64(5))
    for _ in range(3):  # three epochs' permutations before the "interruption"
        assert np.array_equal(rng.permutation(1000), ref.permutation(1000))
    sel.save_checkpoint(path, prm, m, v, 123, 3, rng.bit_generator.state, [2.0, 1.5, 1.25], 0, 2e-3)
    ck = sel.load_checkpoint(path)
    assert np.array_equal(ck["params"], prm) and np.array_equal(ck["m"], m) and np.array_equal(ck["v"], v)
    assert (ck["step"], ck["epoch"], ck["hist"], ck["seed"], ck["lr"]) == (123, 3, [2.0, 1.5, 1.25], 0, 2e-3)
    resumed = np.random.Generator(np.random.PCG64(0))
    resumed.bit_generator.state = ck["rng"]
    for _ in range(3):  # the next epochs shuffle exactly as without the interruption
        assert np.array_equal(resumed.permutation(1000), ref.permutation(1000))


def test_interrupted_write_keeps_previous_checkpoint(tmp_path, monkeypatch):
    path = str(tmp_path / "sel.ckpt")
    prm, m, v = state(2)
    st = np.random.Generator(np.random.PCG64(0)).bit_generator.state
    sel.save_checkpoint(path, prm, m, v, 10, 1, st, [1.0], 0, 1e-3)

    def fail(*a, **k):
        raise OSError("disk full")

    monkeypatch.setattr(np, "savez", fail)
    with pytest.raises(OSError):
        sel.save_checkpoint(path, prm + 1, m, v, 20, 2, st, [1.0, 0.5], 0, 1e-3)
    ck = sel.load_checkpoint(path)
    assert ck["epoch"] == 1 and np.array_equal(ck["params"], prm)
    assert os.listdir(tmp_path) == ["sel.ckpt"]  # no partial file left behind


@pytest.mark.parametrize("field,value", [("version", 99), ("n_param", SEL_NPARAM + 1)])
def test_refuses_other_format(tmp_path, field, value):
    path = str(tmp_path / "sel.ckpt")
    prm, m, v = state(3)
    st = np.random.Generator(np.random.PCG64(0)).bit_generator.state
    sel.save_checkpoint(path, prm, m, v, 1, 1, st, [1.0], 0, 1e-3)
    with np.load(path) as z:
        arrs = {k: np.array(z[k]) for k in z.files}
    meta = json.loads(bytes(arrs["meta"]).decode())
    meta[field] = value
    arrs["meta"] = np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8)
    with open(path, "wb") as fh:
        np.savez(fh, **arrs)
    with pytest.raises(ValueError):
        sel.load_checkpoint(path)
