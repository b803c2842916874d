"""Selector checkpoints round-trip (CPU): parameters bit for bit, target scaling and
loss history; a file of the wrong size is refused."""
import numpy as np
import pytest

from paper_2004_09350_gb300 import morphstore as ms
from paper_2004_09350_gb300 import selector


def test_save_load_round_trip(tmp_path):
    sel = selector.Selector("cpu", seed=3)
    sel.mu = np.arange(10, dtype=np.float32)
    sel.sd = np.linspace(1, 2, 10).astype(np.float32)
    sel.loss_history = [(1, 0.5), (20, 0.25)]
    prefix = str(tmp_path / "sel")
    sel.save(prefix)
    got = selector.Selector.load(prefix, "cpu")
    assert got.params.numel() == ms.MLP_PARAMS
    np.testing.assert_array_equal(got.params.numpy(), sel.params.numpy())
    np.testing.assert_array_equal(got.mu, sel.mu)
    np.testing.assert_array_equal(got.sd, sel.sd)
    assert got.loss_history == sel.loss_history


def test_wrong_size_is_refused(tmp_path):
    sel = selector.Selector("cpu")
    prefix = str(tmp_path / "sel")
    sel.save(prefix)
    np.zeros(10, dtype="<f4").tofile(prefix + ".bin")
    with pytest.raises(ValueError):
        selector.Selector.load(prefix, "cpu")
