"""bench.py reports the blend's captured DRAM traffic only for the kernel
sources it was captured on: the figure carries a SHA-256 prefix of the
blend's sources (render.cu, then clod_internal.cuh), and any other prefix
gives null."""
import hashlib
import os


def _prefix(bench):
    h = hashlib.sha256()
    base = os.path.join(os.path.dirname(os.path.abspath(bench.__file__)), "paper_2510_09997_gb300", "csrc")
    for f in ("render.cu", "clod_internal.cuh"):
        with open(os.path.join(base, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def test_traffic_reported_only_for_the_captured_sources(monkeypatch):
    import bench
    rec = dict(bench.BLEND_TRAFFIC)
    assert rec["bytes_per_launch"] == rec["read"] + rec["write"]
    monkeypatch.setitem(bench.BLEND_TRAFFIC, "sources", _prefix(bench))
    assert bench.blend_traffic() == rec["bytes_per_launch"]
    other = "0" * 16 if _prefix(bench) != "0" * 16 else "1" * 16
    monkeypatch.setitem(bench.BLEND_TRAFFIC, "sources", other)
    assert bench.blend_traffic() is None
