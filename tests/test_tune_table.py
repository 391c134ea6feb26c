"""The tuning table of the C ABI (host-only calls, no GPU): keys, the L
class, validation, and the save / load file format."""
import os

import pytest

SMS = 152


@pytest.fixture()
def sp():
    from paper_0908_3252_gb300 import build, spirec
    build.build()
    spirec.load()
    spirec.spirec_tune_clear()
    yield spirec
    spirec.spirec_tune_clear()  # the table is process-wide: leave it empty


def test_set_get_count_clear(sp):
    G, D, LR = sp.SPIREC_KNOB_GRAM_SPLIT, sp.SPIREC_KNOB_ADJOINT_SPLIT, sp.SPIREC_KNOB_LOOP_ROWS
    sp.spirec_tune_set(G, 64, 128, 1, 4096, 38, sms=SMS)
    sp.spirec_tune_set(D, 64, 128, 1, 4096, 19, sms=SMS)
    sp.spirec_tune_set(LR, 64, 128, 1, 4096, 32, sms=SMS)
    assert sp.spirec_tune_count() == 3
    assert sp.spirec_tune_get(G, 64, 128, 1, 4096, sms=SMS) == 38
    assert sp.spirec_tune_get(D, 64, 128, 1, 4096, sms=SMS) == 19
    # every key field separates entries
    assert sp.spirec_tune_get(G, 64, 128, 2, 4096, sms=SMS) == 0
    assert sp.spirec_tune_get(G, 64, 256, 1, 4096, sms=SMS) == 0
    assert sp.spirec_tune_get(G, 65, 129, 1, 4096, sms=SMS) == 0
    assert sp.spirec_tune_get(G, 64, 128, 1, 4096, sms=SMS + 1) == 0
    sp.spirec_tune_set(G, 64, 128, 1, 4096, 0, sms=SMS)  # 0 removes
    assert sp.spirec_tune_get(G, 64, 128, 1, 4096, sms=SMS) == 0
    assert sp.spirec_tune_count() == 2
    sp.spirec_tune_clear()
    assert sp.spirec_tune_count() == 0


def test_l_class_and_loop_key(sp):
    """Contraction keys share an entry over L in (2^(c-1), 2^c]; the loop's
    key ignores L."""
    G, LR = sp.SPIREC_KNOB_GRAM_SPLIT, sp.SPIREC_KNOB_LOOP_ROWS
    sp.spirec_tune_set(G, 32, 64, 0, 1000, 7, sms=SMS)
    assert sp.spirec_tune_get(G, 32, 64, 0, 513, sms=SMS) == 7
    assert sp.spirec_tune_get(G, 32, 64, 0, 1024, sms=SMS) == 7
    assert sp.spirec_tune_get(G, 32, 64, 0, 512, sms=SMS) == 0
    assert sp.spirec_tune_get(G, 32, 64, 0, 1025, sms=SMS) == 0
    sp.spirec_tune_set(LR, 32, 64, 0, 1000, 16, sms=SMS)
    assert sp.spirec_tune_get(LR, 32, 64, 0, 1, sms=SMS) == 16
    assert sp.spirec_tune_get(LR, 32, 64, 0, 10 ** 9, sms=SMS) == 16


def test_tile_knobs_round_trip(sp):
    """The tile-shape knobs are keyed like the split knobs (by L class)."""
    GT, DT = sp.SPIREC_KNOB_GRAM_TILE, sp.SPIREC_KNOB_ADJOINT_TILE
    assert sp.SPIREC_NUM_KNOBS == 5
    sp.spirec_tune_set(GT, 256, 512, 1, 5000, 2, sms=SMS)
    sp.spirec_tune_set(DT, 256, 512, 2, 5000, 1, sms=SMS)
    assert sp.spirec_tune_get(GT, 256, 512, 1, 8192, sms=SMS) == 2  # the same L class
    assert sp.spirec_tune_get(GT, 256, 512, 1, 8193, sms=SMS) == 0
    assert sp.spirec_tune_get(DT, 256, 512, 2, 5000, sms=SMS) == 1
    assert sp.spirec_tune_get(DT, 256, 512, 1, 5000, sms=SMS) == 0


@pytest.mark.parametrize("args", [
    (5, 32, 64, 0, 100, 1),      # unknown knob (SPIREC_NUM_KNOBS)
    (-1, 32, 64, 0, 100, 1),
    (0, 32, 64, 3, 100, 1),      # unknown precision
    (0, 1, 64, 0, 100, 1),       # N < 2
    (0, 32, 62, 0, 100, 1),      # M < 2N - 1
    (0, 32, 64, 0, 0, 1),        # L < 1
    (0, 32, 64, 0, 100, -1),     # value < 0
])
def test_bad_keys_are_rejected(sp, args):
    knob, N, M, prec, L, value = args
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_tune_set(knob, N, M, prec, L, value, sms=SMS)
    assert e.value.code == sp.SPIREC_EINVAL
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_tune_set(0, 32, 64, 0, 100, 1, sms=-1)
    assert e.value.code == sp.SPIREC_EINVAL
    assert sp.spirec_tune_count() == 0


def test_save_load_round_trip(sp, tmp_path):
    entries = [(0, 64, 128, 1, 4096, 38), (1, 64, 128, 1, 4096, 19), (2, 64, 128, 1, 4096, 32),
               (0, 512, 1024, 2, 131072, 152), (1, 100, 256, 0, 5000, 12)]
    for k, N, M, p, L, v in entries:
        sp.spirec_tune_set(k, N, M, p, L, v, sms=SMS)
    path = str(tmp_path / "tune.txt")
    sp.spirec_tune_save(path)
    lines = open(path).read().splitlines()
    assert lines[0] == "spirec-tune 1" and len(lines) == 1 + len(entries)
    sp.spirec_tune_clear()
    sp.spirec_tune_load(path)
    assert sp.spirec_tune_count() == len(entries)
    for k, N, M, p, L, v in entries:
        assert sp.spirec_tune_get(k, N, M, p, L, sms=SMS) == v
    # a load adds to the table and replaces equal keys
    sp.spirec_tune_set(0, 64, 128, 1, 4096, 5, sms=SMS)
    sp.spirec_tune_set(0, 80, 160, 1, 4096, 6, sms=SMS)
    sp.spirec_tune_load(path)
    assert sp.spirec_tune_get(0, 64, 128, 1, 4096, sms=SMS) == 38
    assert sp.spirec_tune_get(0, 80, 160, 1, 4096, sms=SMS) == 6


@pytest.mark.parametrize("body", [
    "",                                            # empty file
    "spirec-tune 2\n0 64 128 1 12 152 38\n",        # other format
    "spirec-tune 1\n0 64 128 1 12 152\n",          # field missing
    "spirec-tune 1\n0 64 128 1 12 152 38 4\n",     # field too many
    "spirec-tune 1\n0 64 128 1 12 152 x\n",        # not a number
    "spirec-tune 1\n0 64 128 1 12 152 0\n",        # value 0
    "spirec-tune 1\n0 64 128 1 12 0 38\n",         # sms 0
    "spirec-tune 1\n2 64 128 1 12 152 32\n",       # loop key with an L class
    "spirec-tune 1\n0 64 100 1 12 152 38\n",       # M < 2N - 1
    "spirec-tune 1\n0 64 128 1 12 152 38\n9 64 128 1 12 152 38\n",  # bad second line
])
def test_bad_files_leave_the_table_unchanged(sp, tmp_path, body):
    sp.spirec_tune_set(1, 48, 96, 0, 2000, 3, sms=SMS)
    path = tmp_path / "bad.txt"
    path.write_text(body)
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_tune_load(str(path))
    assert e.value.code == sp.SPIREC_EINVAL
    assert sp.spirec_tune_count() == 1
    assert sp.spirec_tune_get(1, 48, 96, 0, 2000, sms=SMS) == 3


def test_missing_file_and_unwritable_path(sp, tmp_path):
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_tune_load(str(tmp_path / "absent.txt"))
    assert e.value.code == sp.SPIREC_EINVAL
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_tune_save(os.path.join(str(tmp_path), "no_such_dir", "t.txt"))
    assert e.value.code == sp.SPIREC_EINVAL
