"""Host logic of bench.py that decides what the JSON line may claim: the kernel-source
hash that ties the committed ncu traffic figure to the code it was measured on."""
import os

import bench


def _write(root, text):
    d = os.path.join(root, "k")
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(d, "a.cu"), "w") as f:
        f.write(text)
    return ["k/a.cu"]


def test_source_hash_ignores_comments_and_spacing(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    paths = _write(str(tmp_path), "int f(int a) {\n  return a + 1;  // add one\n}\n/* note */\n")
    h0 = bench.source_hash(paths)
    _write(str(tmp_path), "int f(int a) {   return a + 1; // reworded comment\n}\n")
    assert bench.source_hash(paths) == h0
    _write(str(tmp_path), "int f(int a) {\n  return a + 2;\n}\n")
    assert bench.source_hash(paths) != h0


def test_traffic_only_while_the_profile_matches_the_code(tmp_path, monkeypatch):
    """The committed profile's DRAM bytes are reported only while its recorded hash is
    the hash of the current kernel sources."""
    real = bench.traffic_from_profiles("n2m")
    if real is not None:
        assert real > 0
    monkeypatch.setattr(bench, "FORCE_SOURCES", ["bench.py"])
    assert bench.traffic_from_profiles("n2m") is None
