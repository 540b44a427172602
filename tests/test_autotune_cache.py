"""Host logic of the autotuning cache (CPU only; the C calls are faked)."""
import json

from paper_2511_22468_gb300 import autotune


class FakeNB:
    def __init__(self):
        self.calls = []

    def nbody_autotune(self, h, probe):
        self.calls.append(("tune", probe))
        return 5, [1.0] * 8

    def nbody_set_tuning(self, h, c):
        self.calls.append(("set", c))


def test_cache_roundtrip(tmp_path, monkeypatch):
    fake = FakeNB()
    monkeypatch.setattr(autotune, "nb", fake)
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "at.json"))
    c, src, ms = autotune.tune(None, [2048, 5000, 32768], "GPU-X", probe_steps=2)
    assert (c, src) == (5, "measured") and fake.calls == [("tune", 2)]
    # same GPU and padded shape (5000 and 5100 pad alike): cached
    c, src, ms = autotune.tune(None, [5100, 32768, 2048], "GPU-X")
    assert (c, src, ms) == (5, "cache", None) and fake.calls[-1] == ("set", 5)
    # another GPU: measured again
    autotune.tune(None, [2048, 5000, 32768], "GPU-Y")
    assert fake.calls[-1] == ("tune", 3)
    db = json.load(open(tmp_path / "at.json"))
    assert len(db) == 2
