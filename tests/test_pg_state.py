"""Checkpoint and resume of the projected-gradient state (host side): x, the
steps done, the step size and the last f values round-trip through an .npz,
and a mismatched x or step size is refused."""
import numpy as np
import pytest
import torch

import paper_2103_09683_gb300 as dose


def test_pg_state_round_trip(tmp_path):
    x = torch.from_numpy(np.random.default_rng(1).uniform(0, 1, 500).astype(np.float32))
    f = torch.linspace(10.0, 1.0, 100, dtype=torch.float64)
    path = str(tmp_path / "pg.npz")
    dose.save_pg_state(path, x, 300, 2.5e-9, f)
    y = torch.zeros(500)
    ptr = y.data_ptr()
    steps, fh = dose.load_pg_state(path, y, 2.5e-9)
    assert steps == 300 and torch.equal(y, x) and y.data_ptr() == ptr  # in place
    assert np.array_equal(fh, f.numpy())


def test_pg_state_refuses_a_mismatch(tmp_path):
    path = str(tmp_path / "pg.npz")
    dose.save_pg_state(path, torch.ones(10), 5, 1e-3)
    with pytest.raises(ValueError, match="spot weights"):
        dose.load_pg_state(path, torch.zeros(11))
    with pytest.raises(ValueError, match="eta"):
        dose.load_pg_state(path, torch.zeros(10), 2e-3)
    steps, fh = dose.load_pg_state(path, torch.zeros(10))
    assert steps == 5 and fh.size == 0
