"""Host logic of the block-length tuner (no GPU): rules from measurements,
the library's use of a rule table, and the committed cache's form."""
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


def test_rules_follow_the_fastest_length_with_geometric_switches():
    meas = {1024: {4: 1.0, 8: 2.0, 16: 3.0, 32: 4.0},
            65536: {4: 1.0, 8: 1.1, 16: 1.5, 32: 2.0},
            262144: {4: 3.0, 8: 2.0, 16: 2.1, 32: 2.5},
            1 << 20: {4: 9.0, 8: 5.0, 16: 3.0, 32: 2.9},
            1 << 22: {4: 30.0, 8: 20.0, 16: 11.0, 32: 10.0}}
    rules = tune.rules_from(meas)
    assert rules == [(131072, 4), (524288, 8), (tune.T_NEVER, 32)]
    for T, row in meas.items():
        assert tune.choose(rules, T) == min(row, key=row.get)
    assert tune.choose(rules, 131071) == 4 and tune.choose(rules, 131072) == 8


def test_noise_within_the_hysteresis_keeps_the_previous_choice():
    meas = {1000: {4: 1.0, 8: 1.2, 16: 2.0, 32: 3.0},
            2000: {4: 1.01, 8: 1.0, 16: 2.0, 32: 3.0},      # 8 faster by 1 %: keep 4
            4000: {4: 1.5, 8: 1.0, 16: 1.01, 32: 3.0},      # 8 clearly faster
            8000: {4: 3.0, 8: 1.0, 16: 0.995, 32: 3.0}}     # 16 faster by 0.5 %: keep 8
    assert tune.rules_from(meas) == [(2829, 4), (tune.T_NEVER, 8)]


def test_ties_go_to_the_shorter_block_and_one_size_gives_one_rule():
    assert tune.rules_from({5000: {4: 1.0, 8: 1.0, 16: 2.0, 32: 3.0}}) == [(tune.T_NEVER, 4)]
    assert tune.rules_from({}) == []


def test_library_uses_the_rules_it_is_given(ks):
    for nx in tune.SLOTS:
        ks.set_chunk_rules(nx, [])
        for T in (1, 1000, 98303, 98304, 196608, 655359, 655360, 1 << 22):
            assert ks.chunk_steps(nx, T) == tune.builtin(T)
    rules = [(5000, 32), (70000, 8), (tune.T_NEVER, 16)]
    ks.set_chunk_rules(4, rules)
    for T in (1, 4999, 5000, 69999, 70000, 1 << 30):
        assert ks.chunk_steps(4, T) == tune.choose(rules, T)
    assert ks.chunk_steps(2, 1000) == tune.builtin(1000)      # other sizes keep their tables
    ks.set_chunk_rules(4, [])
    assert ks.chunk_steps(4, 4999) == 4
    assert ks.chunk_steps(5, 1000) == 0


@pytest.mark.parametrize("rules", [[(100, 5)], [(100, 4), (100, 8)], [(200, 4), (100, 8)], [(0, 4)],
                                   [(i + 1, 4) for i in range(17)]])
def test_malformed_rules_are_rejected(ks, rules):
    with pytest.raises(ks.KsError) as ei:
        ks.set_chunk_rules(4, rules)
    assert ei.value.code == ks.KS_EINVAL
    with pytest.raises(ks.KsError):
        ks.set_chunk_rules(3, [(100, 4)])


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
            assert rules and all(s in tune.STEPS for _, s in rules)
            tbs = [tb for tb, _ in rules]
            assert tbs == sorted(tbs) and len(set(tbs)) == len(tbs)
            # at every measured size the rules pick a length within the hysteresis of the fastest
            meas = {int(T): {int(s): ms for s, ms in row.items()} for T, row in d["measured_ms"][key].items()}
            for T, row in meas.items():
                assert row[tune.choose(rules, T)] <= (1 + tune.HYSTERESIS) * min(row.values()) + 1e-9
