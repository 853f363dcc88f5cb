"""Graph files (.rng binary edge lists and DIMACS .gr text): parsing on the CPU, and a
graph loaded from a file answering like the same graph loaded from arrays (GPU)."""
import numpy as np
import pytest

from paper_1607_07696_gb300 import inputs as I


@pytest.fixture(scope="module")
def rn():
    from paper_1607_07696_gb300 import build as B

    B.build()
    from paper_1607_07696_gb300 import rn as RN

    return RN


def test_rng_round_trip(rn, tmp_path):
    e = I.road_graph(2000, 5540, 3)
    path = str(tmp_path / "g.rng")
    rn.rn_graph_write_file(path, e.src, e.dst, e.w, e.n, rn.RN_UNDIRECTED | rn.RN_REORDER)
    n, flags, src, dst, w = rn.rn_file_read(path)
    assert n == e.n and flags == rn.RN_UNDIRECTED | rn.RN_REORDER
    assert np.array_equal(src, e.src) and np.array_equal(dst, e.dst) and np.array_equal(w, e.w)
    # an empty graph too
    rn.rn_graph_write_file(path, [], [], [], 5, 0)
    assert rn.rn_file_read(path)[:2] == (5, 0) and len(rn.rn_file_read(path)[2]) == 0


def test_dimacs(rn, tmp_path):
    path = tmp_path / "g.gr"
    path.write_text("c a tiny road network\nc\np sp 4 5\na 1 2 7\na 2 1 7\na 2 3 4\n\na 3 4 1\na 4 1 9\n")
    n, flags, src, dst, w = rn.rn_file_read(str(path))
    assert n == 4 and flags == rn.RN_REORDER
    assert src.tolist() == [0, 1, 1, 2, 3] and dst.tolist() == [1, 0, 2, 3, 0] and w.tolist() == [7, 7, 4, 1, 9]


@pytest.mark.parametrize("text,what", [
    ("a 1 2 3\n", "after the 'p' line"),
    ("p sp 3 1\na 1 4 2\n", "outside 1..n"),
    ("p sp 3 2\na 1 2 2\n", "the header says"),
    ("p sp 3 1\nx 1 2\n", "unknown line"),
    ("p sp 3 1\np sp 3 1\na 1 2 1\n", "one 'p sp n m' line"),
    ("c nothing\n", "no 'p sp n m' line"),
])
def test_dimacs_errors(rn, tmp_path, text, what):
    path = tmp_path / "bad.gr"
    path.write_text(text)
    with pytest.raises(rn.RNError) as ex:
        rn.rn_file_read(str(path))
    assert ex.value.status == rn.RN_EINVAL and what in str(ex.value), str(ex.value)


def test_rng_errors(rn, tmp_path):
    e = I.path_graph([1, 2, 3])
    path = tmp_path / "g.rng"
    rn.rn_graph_write_file(str(path), e.src, e.dst, e.w, e.n)
    data = path.read_bytes()
    (tmp_path / "short.rng").write_bytes(data[:-4])
    with pytest.raises(rn.RNError) as ex:
        rn.rn_file_read(str(tmp_path / "short.rng"))
    assert "size does not match m" in str(ex.value)
    bad_flags = bytearray(data)
    bad_flags[8] = 0x80
    (tmp_path / "flags.rng").write_bytes(bytes(bad_flags))
    with pytest.raises(rn.RNError) as ex:
        rn.rn_file_read(str(tmp_path / "flags.rng"))
    assert "unknown flags" in str(ex.value)
    with pytest.raises(rn.RNError) as ex:
        rn.rn_file_read(str(tmp_path / "missing.rng"))
    assert "cannot open" in str(ex.value)
    with pytest.raises(rn.RNError):
        rn.rn_graph_write_file(str(tmp_path / "f.rng"), [0], [1], [1], 2, 0x40)


@pytest.mark.gpu
def test_load_file_answers_like_arrays(rn, oracle, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = I.road_graph(20_000, 55_400, 13)
    path = str(tmp_path / "g.rng")
    rn.rn_graph_write_file(path, e.src, e.dst, e.w, e.n)
    g = rn.rn_graph_load_file(path)
    assert g.n == e.n
    R, S = I.disjoint_sets(e.n, 300, 400, 14)
    ref = oracle.graph(e.n, e.src, e.dst, e.w).join(R, S, 40_000)
    u, v, d = rn.rn_distance_join(g, R, S, 40_000)
    assert np.array_equal(u, ref.u) and np.array_equal(v, ref.v) and np.array_equal(d.astype(np.uint64), ref.d)
    # the DIMACS form of the same roads (both directions of every edge)
    gr = tmp_path / "g.gr"
    lines = [f"p sp {e.n} {2 * e.m}"]
    for a, b, w in zip(e.src.tolist(), e.dst.tolist(), e.w.tolist()):
        lines += [f"a {a + 1} {b + 1} {w}", f"a {b + 1} {a + 1} {w}"]
    gr.write_text("\n".join(lines) + "\n")
    g2 = rn.rn_graph_load_file(str(gr))
    u2, v2, d2 = rn.rn_distance_join(g2, R, S, 40_000)
    assert np.array_equal(u2, ref.u) and np.array_equal(v2, ref.v) and np.array_equal(d2.astype(np.uint64), ref.d)
