"""Host logic of the batch autotuner (no GPU): the signature, the choice of the fastest
candidate, the on-disk record and its reuse."""
import json

import workloads as wl
from paper_1603_06855_gb300 import autotune


def small_batch():
    return [d for d in wl.batch32_mixed()[:6]]


def test_signature_depends_on_the_batch_and_the_gpu():
    ds = small_batch()
    s0 = autotune.signature(ds, 1, "GB300", 152)
    assert s0 == autotune.signature(list(reversed(ds)), 1, "GB300", 152)  # order-free
    assert s0 != autotune.signature(ds[:-1], 1, "GB300", 152)
    assert s0 != autotune.signature(ds, 0, "GB300", 152)
    assert s0 != autotune.signature(ds, 1, "GB300", 148)


def test_tune_records_the_fastest_and_choose_reuses_it(tmp_path):
    ds = small_batch()
    path = str(tmp_path / "rec.json")
    times = {(1, 0): 3.0, (2, 0): 2.0, (4, 0): 1.5, (8, 0): 1.5, (4, 1): 1.7, (8, 1): 2.5, (16, 1): 2.6}
    calls = []

    def fake_measure(designs, precision, rhos, w, g):
        calls.append((w, g))
        return times[(w, g)]

    assert autotune.choose(ds, 1, None, fake_measure, "GB300", 152, path) == (4, 0)  # tie -> fewer workers
    assert sorted(calls) == sorted(times)
    rec = json.load(open(path))
    (entry,) = rec.values()
    assert entry["choice"] == [4, 0] and entry["seconds"]["8,1"] == 2.5
    calls.clear()
    assert autotune.choose(ds, 1, None, fake_measure, "GB300", 152, path) == (4, 0)
    assert calls == []  # recorded: no measurement
    # a different batch is tuned separately, in the same file
    autotune.choose(ds[:3], 1, None, fake_measure, "GB300", 152, path)
    assert len(json.load(open(path))) == 2
