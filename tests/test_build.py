"""The in-tree build reuses a library only when it was built from the current
sources and flags on this machine type (no GPU needed)."""
import os

from paper_1005_4713_gb300 import build as bld


def _point_at(tmp_path, monkeypatch):
    lib = tmp_path / "libspkmc.so"
    monkeypatch.setattr(bld, "LIB", str(lib))
    monkeypatch.setattr(bld, "STAMP", str(lib) + ".sha256")
    return lib


def test_source_hash_is_stable_and_covers_every_input():
    h = bld.source_hash()
    assert h == bld.source_hash() and len(h) == 64
    for name in bld.SOURCES + bld.HEADERS:
        assert os.path.exists(os.path.normpath(os.path.join(bld.CSRC, name))), name


def test_a_library_without_a_matching_stamp_is_rebuilt(tmp_path, monkeypatch):
    lib = _point_at(tmp_path, monkeypatch)
    assert bld._stale()                       # nothing there
    lib.write_bytes(b"not built here")
    assert bld._stale()                       # a library with no stamp (copied in, or pushed)
    (tmp_path / "libspkmc.so.sha256").write_text("0" * 64 + "\n")
    assert bld._stale()                       # built from other sources
    (tmp_path / "libspkmc.so.sha256").write_text(bld.source_hash() + "\n")
    assert not bld._stale()                   # built from these


def test_the_hash_follows_the_flags_and_the_machine(monkeypatch):
    h = bld.source_hash()
    monkeypatch.setattr(bld, "NVCC_FLAGS", bld.NVCC_FLAGS + ["-DX"])
    assert bld.source_hash() != h
    monkeypatch.undo()
    monkeypatch.setattr(bld.platform, "machine", lambda: "some-other-arch")
    assert bld.source_hash() != h
