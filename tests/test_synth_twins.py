"""The GPU-side generators (int64 torch arithmetic) reproduce the numpy SplitMix64
streams bit for bit, run here on the CPU: the bench builds its columns on the
device, and the oracle checks them from the numpy twins."""
import numpy as np
import torch

from paper_2004_09350_gb300 import synth


def bits(t):
    return t.numpy().view(np.uint64)


def test_splitmix_and_uniform_twins():
    for seed in (0, 1, 2**63 + 5):
        np.testing.assert_array_equal(bits(synth.splitmix64_torch(seed, 1000, "cpu")), synth.splitmix64(seed, 1000))
    for lo, hi in ((0, 64), (0, 1 << 40), (7, 2_500_007), (2**62, 2**62 + 64)):
        np.testing.assert_array_equal(bits(synth.uniform_torch(3, 5000, lo, hi, "cpu")), synth.uniform(3, 5000, lo, hi))


def test_skewed_widths_twin():
    for n in (1, 511, 512, 513, 5000):
        for widths in (synth.WIDTH_CHOICES, (1, 5, 40)):
            np.testing.assert_array_equal(bits(synth.skewed_widths_torch(9, n, widths, "cpu")),
                                          synth.skewed_widths(9, n, widths))


def test_star_fact_twin():
    a = synth.star_fact(4, 3000)
    b = synth.star_fact_torch(4, 3000, "cpu")
    for k in a:
        np.testing.assert_array_equal(bits(b[k]), a[k], err_msg=k)


def test_batch_fragment_twins_and_ranges():
    specs = synth.batch_fragments(17, 64, lo_log2=0, hi_log2=13)
    assert {s["shape"] for s in specs} == set(synth.BATCH_Y_SHAPES)
    for sp in specs:
        x, y = synth.batch_x(sp), synth.batch_y(sp)
        assert x.size == y.size == sp["n"]
        np.testing.assert_array_equal(bits(synth.batch_x_torch(sp, "cpu")), x)
        np.testing.assert_array_equal(bits(synth.batch_y_torch(sp, "cpu")), y)
        assert 1 <= sp["bx"] <= 40 and 1 <= sp["by"] <= 40
        if x.size:
            assert int(x.max()) < 1 << sp["bx"]
        if sp["shape"] == "sorted" and y.size:
            assert (np.diff(y.astype(np.int64)) >= 0).all()
        if sp["shape"] in ("uniform", "offset", "skewed") and y.size:
            assert int(y.max()) < 1 << sp["by"]


def test_batch_lengths_are_log_uniform():
    n = np.array([s["n"] for s in synth.batch_fragments(3, 4096)], dtype=np.float64)
    assert n.min() >= 2**10 and n.max() <= 2**24
    # log2 n uniform on [10, 24]: mean 17, and the mean length (2^24 - 2^10) / (14 ln 2) ~ 1.73e6
    assert abs(np.log2(n).mean() - 17.0) < 0.2
    assert 1.5e6 < n.mean() < 2.0e6
