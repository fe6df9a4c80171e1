"""Host logic of the block-length and block-fold tuner (no GPU): rules from
measurements, the library's use of a rule table, and the committed cache's
form."""
import glob
import json
import os

import pytest

from paper_1905_13002_gb300 import tune


@pytest.fixture(scope="module")
def ks():
    from paper_1905_13002_gb300 import _build
    _build.build()
    import paper_1905_13002_gb300 as ks
    yield ks
    for nx in tune.SLOTS:
        ks.set_chunk_rules(nx, [])


def test_rules_follow_the_fastest_variant_with_geometric_switches():
    meas = {1024: {(4, 0): 1.0, (8, 0): 2.0, (16, 0): 3.0, (32, 0): 4.0, (4, 1): 1.5},
            65536: {(4, 0): 1.0, (8, 0): 1.1, (16, 0): 1.5, (32, 0): 2.0, (4, 1): 1.4},
            262144: {(4, 0): 3.0, (8, 0): 2.0, (16, 0): 2.1, (32, 0): 2.5, (8, 1): 2.3},
            1 << 20: {(4, 0): 9.0, (8, 0): 5.0, (16, 0): 3.0, (32, 0): 2.9, (32, 1): 2.7},
            1 << 22: {(4, 0): 30.0, (8, 0): 20.0, (16, 0): 11.0, (32, 0): 10.0, (32, 1): 9.0}}
    rules = tune.rules_from(meas)
    assert rules == [(131072, 4, 0), (524288, 8, 0), (tune.T_NEVER, 32, 1)]
    for T, row in meas.items():
        assert tune.choose(rules, T) == min(row, key=row.get)
    assert tune.choose(rules, 131071) == (4, 0) and tune.choose(rules, 131072) == (8, 0)


def test_noise_within_the_hysteresis_keeps_the_previous_choice():
    meas = {1000: {(4, 0): 1.0, (8, 0): 1.2, (16, 0): 2.0, (32, 0): 3.0},
            2000: {(4, 0): 1.01, (8, 0): 1.0, (16, 0): 2.0, (32, 0): 3.0},     # 8 faster by 1 %: keep 4
            4000: {(4, 0): 1.5, (8, 0): 1.0, (16, 0): 1.01, (8, 1): 1.0},      # 8 clearly faster
            8000: {(4, 0): 3.0, (8, 0): 1.0, (16, 0): 0.995, (8, 1): 0.99}}    # others within 1 %: keep 8
    assert tune.rules_from(meas) == [(2829, 4, 0), (tune.T_NEVER, 8, 0)]


def test_ties_go_to_the_shorter_block_without_the_fold_and_one_size_gives_one_rule():
    assert tune.rules_from({5000: {(4, 1): 1.0, (4, 0): 1.0, (16, 0): 2.0}}) == [(tune.T_NEVER, 4, 0)]
    assert tune.rules_from({}) == []


def test_variant_keys_round_trip():
    for v in tune.VARIANTS:
        assert tune.vparse(tune.vkey(v)) == v
    assert tune.vkey((32, 1)) == "32f" and tune.vkey((8, 0)) == "8"


def test_library_uses_the_rules_it_is_given(ks):
    for nx in tune.SLOTS:
        ks.set_chunk_rules(nx, [])
        for T in (1, 1000, 98303, 98304, 196608, 655359, 655360, 1 << 22):
            assert (ks.chunk_steps(nx, T), ks.chunk_fold(nx, T)) == tune.builtin(T, nx)
    rules = [(5000, 32, 1), (70000, 8, 0), (tune.T_NEVER, 16, 1)]
    ks.set_chunk_rules(4, rules)
    for T in (1, 4999, 5000, 69999, 70000, 1 << 30):
        assert (ks.chunk_steps(4, T), ks.chunk_fold(4, T)) == tune.choose(rules, T)
    assert (ks.chunk_steps(2, 1000), ks.chunk_fold(2, 1000)) == tune.builtin(1000, 2)   # other sizes keep theirs
    ks.set_chunk_rules(4, [])
    assert ks.chunk_steps(4, 4999) == 4 and ks.chunk_fold(4, 1 << 22) == 1 and ks.chunk_fold(0, 1 << 22) == 0
    assert ks.chunk_steps(5, 1000) == 0 and ks.chunk_fold(5, 1 << 22) == 0


@pytest.mark.parametrize("rules", [[(100, 5, 0)], [(100, 4, 0), (100, 8, 0)], [(200, 4, 0), (100, 8, 0)],
                                   [(0, 4, 0)], [(100, 4, 2)], [(100, 4, -1)],
                                   [(i + 1, 4, 0) for i in range(17)]])
def test_malformed_rules_are_rejected(ks, rules):
    with pytest.raises(ks.KsError) as ei:
        ks.set_chunk_rules(4, rules)
    assert ei.value.code == ks.KS_EINVAL
    with pytest.raises(ks.KsError):
        ks.set_chunk_rules(3, [(100, 4, 0)])


def test_cache_validity_check():
    d = {"version": tune.CACHE_VERSION, "device": "GPU X", "library_version": 100, "rules": {"4": [[10, 4]]}}
    assert tune.valid_cache(d, "GPU X", 100)
    assert not tune.valid_cache(d, "GPU Y", 100)
    assert not tune.valid_cache(d, "GPU X", 101)
    assert not tune.valid_cache(dict(d, version=tune.CACHE_VERSION + 1), "GPU X", 100)


def test_committed_caches_are_well_formed():
    for path in glob.glob(os.path.join(tune.TUNING_DIR, "*.json")):
        with open(path) as f:
            d = json.load(f)
        assert d["version"] == tune.CACHE_VERSION
        assert set(d["rules"]) <= {str(s) for s in tune.SLOTS}
        for key, rules in d["rules"].items():
            assert rules and all(s in tune.STEPS and f in (0, 1) for _, s, f in rules)
            tbs = [tb for tb, _, _ in rules]
            assert tbs == sorted(tbs) and len(set(tbs)) == len(tbs)
            # at every measured size the rules pick a variant within the hysteresis of the fastest
            meas = {int(T): {tune.vparse(k): ms for k, ms in row.items()} for T, row in d["measured_ms"][key].items()}
            for T, row in meas.items():
                assert row[tune.choose(rules, T)] <= (1 + tune.HYSTERESIS) * min(row.values()) + 1e-9
