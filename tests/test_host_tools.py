"""Host-side tools that need no GPU: the autotuner's plan cache file and the stats log."""
import pytest


@pytest.fixture(scope="module")
def rn():
    from paper_1607_07696_gb300 import build as B

    B.build()
    from paper_1607_07696_gb300 import rn as RN

    return RN


def test_tune_cache_round_trip(rn, tmp_path):
    src = tmp_path / "plans.txt"
    src.write_text("rn-tune 1\n70914 32 4 1\n70915 64 8 2\n1245199 128 16 1\n")
    assert rn.rn_tune_cache_load(str(src)) == 3
    out = tmp_path / "saved.txt"
    rn.rn_tune_cache_save(str(out))
    saved = out.read_text().splitlines()
    assert saved[0] == "rn-tune 1"
    assert {"70914 32 4 1", "70915 64 8 2", "1245199 128 16 1"} <= set(saved[1:])


@pytest.mark.parametrize("text,what", [
    ("", "empty file"),
    ("nonsense\n", "not a tune cache"),
    ("rn-tune 1\n5 48 4 1\n", "line 2"),
    ("rn-tune 1\n5 32 0 1\n", "line 2"),
    ("rn-tune 1\n5 32 4 64\n", "line 2"),
])
def test_tune_cache_rejects(rn, tmp_path, text, what):
    p = tmp_path / "bad.txt"
    p.write_text(text)
    with pytest.raises(rn.RNError) as ex:
        rn.rn_tune_cache_load(str(p))
    assert ex.value.status == rn.RN_EINVAL and what in str(ex.value)
    with pytest.raises(rn.RNError):
        rn.rn_tune_cache_load(str(tmp_path / "missing.txt"))
