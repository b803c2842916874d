"""Host logic of the batch autotuner, on the CPU: the candidate list obeys the
launch rules of ms_batch_run, and tune() returns the fastest candidate and serves
it from its cache the second time (timings faked, no GPU)."""
import json

import pytest

from paper_2004_09350_gb300 import autotune
from paper_2004_09350_gb300 import morphstore as ms


def accepted(w, d, t, k, c, s):
    """ms_batch_run's checks on a configuration (mirrored here to pin the list)."""
    lt = t.bit_length() - 1
    if t != 1 << lt or not 3 <= lt <= 10 or c > 1:
        return False
    if s == 0:
        return t >= 2 * d
    if s == 1:
        return c == 0 and t >= w
    if s == 2:
        return c == 0 and w == 8
    return False


def test_candidates_are_all_launchable_and_cover_every_variant():
    cands = autotune.candidates()
    assert cands and len(set(cands)) == len(cands)
    assert all(accepted(*cfg) for cfg in cands)
    assert {(w, d, c, s) for (w, d, t, k, c, s) in cands} == set(ms.BATCH_VARIANTS)
    assert {cfg[5] for cfg in cands} == {0, 1, 2}


def test_tune_picks_the_fastest_and_caches_it(tmp_path, monkeypatch):
    monkeypatch.setenv("MS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(autotune, "signature", lambda batch, device: "dev/152sm/f4/r2^20/b9.0")
    cands = autotune.candidates()
    fake = {cfg: 10.0 + i for i, cfg in enumerate(cands)}
    best_cfg = cands[len(cands) // 2]
    fake[best_cfg] = 1.5
    calls = []

    def timing(batch, sums, cfg, reps=3, stream=None):
        calls.append(cfg)
        return fake[tuple(cfg)]

    monkeypatch.setattr(autotune, "time_config", timing)

    class Sums:
        device = "cpu"

    best, table = autotune.tune(object(), Sums())
    assert best == best_cfg and len(table) == len(cands) and len(calls) == len(cands)
    cached = json.loads((tmp_path / "tune.json").read_text())
    assert cached["dev/152sm/f4/r2^20/b9.0"]["cfg"] == list(best_cfg)
    again, table2 = autotune.tune(object(), Sums())
    assert again == best_cfg and table2 == {best_cfg: 1.5} and len(calls) == len(cands)


def test_tune_skips_variants_that_do_not_fit_and_raises_on_other_errors(tmp_path, monkeypatch):
    monkeypatch.setenv("MS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(autotune, "signature", lambda batch, device: "k")
    cands = autotune.candidates()[:3]

    def too_big(batch, sums, cfg, reps=3, stream=None):
        if cfg == cands[0]:
            raise ms.MSError(ms.MS_ERR_INVALID_ARG, "ms_batch_run")
        return 2.0 if cfg == cands[1] else 3.0

    monkeypatch.setattr(autotune, "time_config", too_big)

    class Sums:
        device = "cpu"

    best, table = autotune.tune(object(), Sums(), cands=cands, use_cache=False)
    assert best == cands[1] and cands[0] not in table

    def broken(batch, sums, cfg, reps=3, stream=None):
        raise ms.MSError(ms.MS_ERR_FORMAT, "ms_batch_run")

    monkeypatch.setattr(autotune, "time_config", broken)
    with pytest.raises(ms.MSError):
        autotune.tune(object(), Sums(), cands=cands, use_cache=False)
