"""The tuning database (gett_tune.h), host only: entries are keyed by the
planned signature -- the Sec. 5.7 arguments after dropping extent-1 modes,
flipping negative increments and fusing stride-compatible modes -- so layouts
that plan to the same canonical problem share an entry and others do not;
files round-trip and a malformed file merges nothing."""
import os

import pytest

from paper_2410_06770_gb300 import gett

# C[a,b,i,j] += A[a,b,c,d] B[c,d,i,j], column-major, small extents
CC = dict(EXTA=(4, 5, 6, 7), INCA=(1, 4, 20, 120), EXTB=(6, 7, 3, 2), INCB=(1, 6, 42, 126),
          CONTA=(2, 3), CONTB=(0, 1), PERM=(0, 1, 2, 3), INCC=(1, 4, 20, 60))


@pytest.fixture(autouse=True)
def _clean():
    from paper_2410_06770_gb300 import build
    build.build()
    gett.tune_db_clear()
    yield
    gett.tune_db_clear()


def with_unit_mode(a):
    """The same problem with an extra extent-1 mode on A (squeezed by the
    planner): A gets a trailing free mode of extent 1 and any increment; it is
    the third free index (A's free modes come first), placed at the last
    output position with any increment."""
    b = dict(a)
    b["EXTA"] = a["EXTA"] + (1,)
    b["INCA"] = a["INCA"] + (999,)
    b["PERM"] = (0, 1, 4, 2, 3)
    b["INCC"] = a["INCC"] + (7,)
    return b


def test_put_get_roundtrip_and_kinds():
    assert gett.tune_db_get(gett.TUNE_SINGLE, "d", CC) is None
    gett.tune_db_put(gett.TUNE_SINGLE, "d", CC, 2, 1, 4)
    assert gett.tune_db_get(gett.TUNE_SINGLE, "d", CC) == (2, 1, 4)
    # kind and operand type are part of the key
    assert gett.tune_db_get(gett.TUNE_BATCH, "d", CC) is None
    assert gett.tune_db_get(gett.TUNE_SINGLE, "s", CC) is None
    gett.tune_db_put(gett.TUNE_SINGLE, "d", CC, 3, 0, 1)  # replaces
    assert gett.tune_db_get(gett.TUNE_SINGLE, "d", CC) == (3, 0, 1)
    assert gett.tune_db_size() == 1


def test_key_is_the_planned_signature():
    gett.tune_db_put(gett.TUNE_BATCH, "f32", CC, 5)
    # an extent-1 mode squeezes away: same entry
    assert gett.tune_db_get(gett.TUNE_BATCH, "f32", with_unit_mode(CC)) == (5, 0, 0)
    # a padded A (other increments) plans differently: no entry
    padded = dict(CC, INCA=(1, 5, 25, 150))
    assert gett.tune_db_get(gett.TUNE_BATCH, "f32", padded) is None
    # the output permutation changes C's increments per class: no entry
    perm = dict(CC, PERM=(1, 0, 2, 3), INCC=(1, 5, 20, 60))
    assert gett.tune_db_get(gett.TUNE_BATCH, "f32", perm) is None


def test_invalid_arguments_report_positions():
    bad = dict(CC, PERM=(0, 0, 2, 3))
    with pytest.raises(gett.GettError) as ei:
        gett.tune_db_put(gett.TUNE_SINGLE, "d", bad, 2)
    assert ei.value.status == gett.GETT_ERR_ARG and ei.value.arg == 12
    with pytest.raises(gett.GettError):
        gett.tune_db_put(7, "d", CC, 2)


def test_save_load_merge(tmp_path):
    gett.tune_db_put(gett.TUNE_SINGLE, "d", CC, 2, 1, 4)
    gett.tune_db_put(gett.TUNE_BATCH, "bf16", CC, 8)
    path = str(tmp_path / "db.txt")
    gett.tune_db_save(path)
    text = open(path).read().splitlines()
    assert text[0].startswith("#") and len(text) == 3
    gett.tune_db_clear()
    assert gett.tune_db_size() == 0
    gett.tune_db_load(path)
    assert gett.tune_db_get(gett.TUNE_SINGLE, "d", CC) == (2, 1, 4)
    assert gett.tune_db_get(gett.TUNE_BATCH, "bf16", CC) == (8, 0, 0)
    # loading merges: a later file replaces an entry and keeps the others
    with open(path, "w") as f:
        f.write(text[0] + "\n" + text[1].rsplit(" ", 3)[0] + " 9 9 9\n")
    gett.tune_db_load(path)
    assert gett.tune_db_size() == 2


def test_malformed_file_merges_nothing(tmp_path):
    path = str(tmp_path / "bad.txt")
    with open(path, "w") as f:
        f.write("1 1 m:4,1,1/n:3,1,1/k:2,1,1/ 2 0 1\n")
        f.write("1 1 only-three-fields\n")
    with pytest.raises(gett.GettError):
        gett.tune_db_load(path)
    assert gett.tune_db_size() == 0
    with pytest.raises(gett.GettError):
        gett.tune_db_load(os.path.join(str(tmp_path), "missing.txt"))
