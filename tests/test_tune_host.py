"""The autotuner's choice and its cache, on the host: the library's variant
calls and the timing are replaced by fakes, so the test needs no GPU.

Checked: the fastest (variant, blocks per SM) wins; a streamed time within
1% of the best wins instead (its time moves less from box to box); the
default is restored before the winner is set, so that a streamed winner keeps
the default grid-stride shape as its fallback; the choice lands in the JSON
cache under the GPU's name and is applied from there by apply(), which skips
variants the library does not compile and entries that are not per format."""
import json

import pytest

from paper_1602_04716_gb300 import tune

STREAMED = 8
RealFormat = tune._b.Format


class FakeLib:
    """Stands in for the binding: compiled variants per (format, op), and a
    record of every bsfp_set_variant call."""

    def __init__(self, compiled):
        self.compiled = compiled
        self.calls = []
        self.VARIANT_STREAMED = STREAMED

    def bsfp_variants_compiled(self, f, op):
        return self.compiled.get((f.exp_bits, f.man_bits, f.rnd, op), [])

    def bsfp_set_variant(self, f, op, wpt, bps):
        self.calls.append((f.exp_bits, f.man_bits, f.rnd, op, wpt, bps))

    @staticmethod
    def Format(e, m, r=0):
        return RealFormat(e, m, r)


@pytest.fixture
def fake(monkeypatch):
    def install(compiled, times):
        lib = FakeLib(compiled)
        monkeypatch.setattr(tune, "_b", lib)
        state = {}

        def fake_time(op, f, a, b, c, out, n, reps=5):
            # the shape last set for (format, op) decides the time
            last = [k for k in lib.calls if k[:4] == (f.exp_bits, f.man_bits, f.rnd, op)][-1]
            state["timed"] = state.get("timed", 0) + 1
            return times[(last[4], last[5])]

        monkeypatch.setattr(tune, "time_op", fake_time)
        monkeypatch.setattr(tune, "gpu_name", lambda: "Fake GPU")
        return lib, state
    return install


F = RealFormat(5, 7, 0)


def test_fastest_shape_wins_and_is_cached(fake, tmp_path):
    lib, state = fake({(5, 7, 0, "mul"): [1, 2, STREAMED]},
                      {(1, 0): 0.30, (1, 4): 0.28, (2, 0): 0.25, (2, 4): 0.21, (STREAMED, 0): 0.24})
    path = str(tmp_path / "cache.json")
    best, table = tune.autotune("mul", F, None, None, None, None, 1 << 20, bps_choices=(0, 4), path=path)
    assert best == (2, 4)
    assert state["timed"] == 5          # two block counts per grid-stride variant, one streamed
    assert lib.calls[-2:] == [(5, 7, 0, "mul", 0, 0), (5, 7, 0, "mul", 2, 4)]   # default first, then the winner
    cache = json.load(open(path))
    assert cache["Fake GPU"]["5/7/0/mul"] == {"wpt": 2, "bps": 4, "ms": 0.21, "n": 1 << 20}


def test_streamed_wins_a_near_tie(fake, tmp_path):
    lib, _ = fake({(5, 7, 0, "add"): [1, 2, STREAMED]},
                  {(1, 0): 0.30, (2, 0): 0.200, (STREAMED, 0): 0.2019})
    best, _ = tune.autotune("add", F, None, None, None, None, 1 << 20, bps_choices=(0,), path=None)
    assert best == (STREAMED, 0)
    assert lib.calls[-2:] == [(5, 7, 0, "add", 0, 0), (5, 7, 0, "add", STREAMED, 0)]


def test_streamed_loses_beyond_one_percent(fake):
    fake({(5, 7, 0, "add"): [1, 2, STREAMED]}, {(1, 0): 0.30, (2, 0): 0.200, (STREAMED, 0): 0.2021})
    best, _ = tune.autotune("add", F, None, None, None, None, 1 << 20, bps_choices=(0,), path=None)
    assert best == (2, 0)


def test_apply_sets_cached_shapes_it_can(fake, tmp_path):
    lib, _ = fake({(5, 7, 0, "mul"): [1, 2, STREAMED], (4, 4, 1, "add"): [1, 2]}, {})
    path = str(tmp_path / "cache.json")
    json.dump({"Fake GPU": {"5/7/0/mul": {"wpt": STREAMED, "bps": 0, "ms": 0.2, "n": 1},
                            "4/4/1/add": {"wpt": 4, "bps": 2, "ms": 0.1, "n": 1},    # 4 not compiled
                            "batch": {"wpt": 2, "bps": 0}},
               "Other GPU": {"4/4/1/add": {"wpt": 2, "bps": 2, "ms": 0.1, "n": 1}}}, open(path, "w"))
    assert tune.apply(path) == 1
    assert lib.calls == [(5, 7, 0, "mul", 0, 0), (5, 7, 0, "mul", STREAMED, 0)]
