"""The stored network weights that bench.py's learned comparison uses: written by learned.train on
the GPU (its kernels) and saved with their training recipe; and the save/load round trip."""
import json

import numpy as np

from paper_1212_6680_gb300 import learned

PATH = "paper_1212_6680_gb300/weights/learned_fpcg_seed5000.npz"


def test_stored_weights_and_recipe():
    w, info = learned.load_weights(PATH)
    assert w.shape == (7776,) and w.dtype == np.float32 and np.all(np.isfinite(w))
    assert info["seed"] == 5000 and info["init_seed"] == 77 and info["nsys"] == 200
    assert info["sides"] == [64, 128] and info["epochs"] == 4 and info["act"] == "bf16"
    assert info["pairs"] > 0 and len(info["loss_per_epoch"]) == 4


def test_save_load_round_trip(tmp_path):
    w = np.random.default_rng(1).standard_normal(7776).astype(np.float32)
    info = {"seed": 3, "note": "x"}
    p = str(tmp_path / "w.npz")
    learned.save_weights(p, w, info)
    w2, i2 = learned.load_weights(p)
    assert np.array_equal(w, w2) and i2 == json.loads(json.dumps(info))
