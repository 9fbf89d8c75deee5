"""Host logic of the schedule switch and the tuning tables (no device needed):
validation, installation, and the lookup that assigns each chain its entry."""
import pytest


@pytest.fixture
def lib(rgflib):
    yield rgflib
    rgflib.set_schedule(rgflib.RGF_SCHED_PHASED)
    rgflib.set_domains(2)
    for p in (rgflib.RGF_FP64, rgflib.RGF_MIXED, rgflib.RGF_MIXED_TC):
        rgflib.set_tuning(p, [])


def test_schedule_switch(lib):
    assert lib.get_schedule() == lib.RGF_SCHED_PHASED
    lib.set_schedule(lib.RGF_SCHED_PERSISTENT)
    assert lib.get_schedule() == lib.RGF_SCHED_PERSISTENT
    with pytest.raises(lib.RGFError):
        lib.set_schedule(7)
    assert lib.get_schedule() == lib.RGF_SCHED_PERSISTENT


def test_default_entry_without_a_table(lib):
    for p in (lib.RGF_FP64, lib.RGF_MIXED, lib.RGF_MIXED_TC):
        assert lib.get_tuning(p) == []
        e = lib.tune_lookup(p, 245)
        assert (e["engine"], e["panel"], e["pairs"]) == (lib.RGF_ENGINE_TENSOR, 0, 1)


def test_lookup_by_column_size(lib):
    table = [dict(K_max=20, engine=0, panel=8, pairs=0),
             dict(K_max=64, engine=1, panel=4, pairs=1),
             dict(K_max=130, engine=1, panel=16, pairs=1)]
    lib.set_tuning(lib.RGF_MIXED_TC, table)
    assert lib.get_tuning(lib.RGF_MIXED_TC) == table
    # K = ceil(N/2): N = 39 -> 20 (first entry), N = 41 -> 21 (second),
    # N = 127 -> 64 (second), N = 129 -> 65 (third), N = 1001 -> beyond: last
    assert lib.tune_lookup(lib.RGF_MIXED_TC, 39) == table[0]
    assert lib.tune_lookup(lib.RGF_MIXED_TC, 41) == table[1]
    assert lib.tune_lookup(lib.RGF_MIXED_TC, 127) == table[1]
    assert lib.tune_lookup(lib.RGF_MIXED_TC, 129) == table[2]
    assert lib.tune_lookup(lib.RGF_MIXED_TC, 1001) == table[2]
    # tables are per precision
    assert lib.get_tuning(lib.RGF_FP64) == []
    lib.set_tuning(lib.RGF_MIXED_TC, [])
    assert lib.get_tuning(lib.RGF_MIXED_TC) == []


@pytest.mark.parametrize("bad", [
    [dict(K_max=0, engine=1, panel=0, pairs=1)],
    [dict(K_max=10, engine=1, panel=0, pairs=1), dict(K_max=10, engine=1, panel=0, pairs=1)],
    [dict(K_max=10, engine=2, panel=0, pairs=1)],
    [dict(K_max=10, engine=1, panel=6, pairs=1)],
    [dict(K_max=10, engine=1, panel=32, pairs=1)],
    [dict(K_max=10, engine=1, panel=0, pairs=2)],
])
def test_invalid_tables_are_refused_and_leave_the_old_one(lib, bad):
    good = [dict(K_max=50, engine=0, panel=8, pairs=1)]
    lib.set_tuning(lib.RGF_MIXED, good)
    with pytest.raises(lib.RGFError) as ei:
        lib.set_tuning(lib.RGF_MIXED, bad)
    assert ei.value.status == lib.RGF_EINVAL
    assert lib.get_tuning(lib.RGF_MIXED) == good


def test_save_and_load_round_trip(lib, tmp_path):
    t2 = [dict(K_max=30, engine=0, panel=16, pairs=1), dict(K_max=300, engine=1, panel=8, pairs=0)]
    t0 = [dict(K_max=99, engine=0, panel=4, pairs=0)]
    lib.set_tuning(lib.RGF_MIXED_TC, t2)
    lib.set_tuning(lib.RGF_FP64, t0)
    f = tmp_path / "tuning.json"
    lib.save_tuning(f)
    for p in (lib.RGF_FP64, lib.RGF_MIXED, lib.RGF_MIXED_TC):
        lib.set_tuning(p, [])
    lib.load_tuning(f)
    assert lib.get_tuning(lib.RGF_MIXED_TC) == t2
    assert lib.get_tuning(lib.RGF_FP64) == t0
    assert lib.get_tuning(lib.RGF_MIXED) == []


def test_autotune_argument_checks(lib):
    with pytest.raises(lib.RGFError):
        lib.autotune(lib.RGF_MIXED_TC, [11, 12], cells=2)     # same column size 6
    with pytest.raises(lib.RGFError):
        lib.autotune(lib.RGF_MIXED_TC, [1], cells=2)
    with pytest.raises(lib.RGFError):
        lib.autotune(lib.RGF_MIXED_TC, [11], cells=0)


def test_automatic_domain_count(lib):
    # one SM per domain for every chain, at most ncol / 32, at least 2, at
    # most ncol / 2
    assert lib.auto_domains(69, 16000, 152) == 2        # the bench batch: two halves
    assert lib.auto_domains(1, 16000, 152) == 152       # one long chain: every SM
    assert lib.auto_domains(10, 16000, 152) == 15
    assert lib.auto_domains(1, 160, 152) == 5
    assert lib.auto_domains(1, 16, 152) == 2
    assert lib.auto_domains(1, 4, 152) == 2
    assert lib.auto_domains(2048, 400, 152) == 2


def test_domain_setting(lib):
    assert lib.get_domains() == 2
    lib.set_domains(7)
    assert lib.get_domains() == 7
    for bad in (1, -2, 5000):
        with pytest.raises(lib.RGFError):
            lib.set_domains(bad)
    assert lib.get_domains() == 7
    lib.set_domains(0)
    assert lib.get_domains() == 0
