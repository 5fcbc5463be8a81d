"""Checkpoint files of a solve's iterate (host logic; no device work)."""

import numpy as np
import torch

from paper_1508_06103_gb300 import api


def test_checkpoint_round_trip_keeps_the_iterate_bit_for_bit(tmp_path):
    x = torch.from_numpy(np.random.default_rng(3).standard_normal(1001))
    path = str(tmp_path / "ckpt.npz")
    api.checkpoint_save(path, x, iterations=17, relres=3.5e-7, restart=30)
    y, meta = api.checkpoint_load(path, device="cpu")
    assert y.dtype == torch.float64 and torch.equal(x, y)
    assert meta == {"iterations": 17, "relres": 3.5e-7, "restart": 30}
