"""Host logic of bench.py's roofline (no GPU): the algorithmic bytes per
event, and the DRAM traffic taken from a committed ncu capture only while the
kernel sources are the ones it was taken on, scaled to the launch's cycles."""
import json
import os

import bench


def test_bytes_per_event():
    # 14 int32 class counts plus the bit-packed block with its one-site halo
    assert bench.bytes_per_event(16) == 14 * 4 + (16 ** 3 + 6 * 16 ** 2) // 8 == 760
    assert bench.bytes_per_event(8) == 56 + (512 + 384) // 8
    # the int8 layout that the bit-packed one is compared with
    assert bench.int8_bytes_per_event(16) == 5632
    # count line + 8 planes + the plane beyond + x, y (2 x 8 words) and z (one face) ghosts of the half
    assert bench.half_domain_floor_bytes(16) == 56 + 256 + 32 + 32 + 32 + 32 == 440


def _write_traffic(root, entry):
    os.makedirs(os.path.join(root, "profiles"))
    with open(os.path.join(root, "profiles", "traffic.json"), "w") as f:
        json.dump({"spkmc-1024^3-d16": entry}, f)


def test_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    assert len(h) == 16
    root = str(tmp_path)
    _write_traffic(root, {"kernel_source_hash": h, "dram_bytes_per_launch": 1000, "cycles_per_launch": 500})
    monkeypatch.setattr(bench, "ROOT", root)
    # the hash is still taken from the package sources, the capture from root
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.ncu_traffic("spkmc-1024^3-d16", 500) == 1000
    assert bench.ncu_traffic("spkmc-1024^3-d16", 250) == 500  # scaled by the cycles
    assert bench.ncu_traffic("spkmc-1024^3-d16", 1000) == 2000
    assert bench.ncu_traffic("another-workload", 500) is None
    # a capture of other kernel sources is not reported
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic("spkmc-1024^3-d16", 500) is None


def test_traffic_without_a_capture(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("spkmc-1024^3-d16", 500) is None


def test_kernel_source_hash_changes_with_the_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1005_4713_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "spkmc_kernels.cu").write_text("a")
    (csrc / "spkmc_device.cuh").write_text("c")
    (csrc / "spkmc_internal.h").write_text("b")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.kernel_source_hash()
    (csrc / "spkmc_kernels.cu").write_text("a1")
    h2 = bench.kernel_source_hash()
    assert h2 != h1
    (csrc / "spkmc_device.cuh").write_text("c1")  # a header the cycle kernel includes
    assert bench.kernel_source_hash() not in (h1, h2)
    # the set-up kernels are another translation unit: not part of the hash
    (csrc / "spkmc_setup_kernels.cu").write_text("d")
    h3 = bench.kernel_source_hash()
    (csrc / "spkmc_setup_kernels.cu").write_text("d1")
    assert bench.kernel_source_hash() == h3


def test_kernel_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1005_4713_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "spkmc_device.cuh").write_text("int c;")
    (csrc / "spkmc_internal.h").write_text("int b;")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    code = 'int a = 1;\nconst char *s = "// not a comment";\n'
    (csrc / "spkmc_kernels.cu").write_text(code)
    h = bench.kernel_source_hash()
    (csrc / "spkmc_kernels.cu").write_text("// a comment\n" + code.replace("1;", "1; /* another */") + "\n\n")
    assert bench.kernel_source_hash() == h
    (csrc / "spkmc_kernels.cu").write_text(code.replace("not a comment", "still not"))
    assert bench.kernel_source_hash() != h  # text inside a string literal is code
    (csrc / "spkmc_kernels.cu").write_text(code.replace("1;", "2;"))
    assert bench.kernel_source_hash() != h


def test_binder_table_bins_by_edge_and_temperature():
    binder = [{"L": 16, "T": 4.41, "U": 0.50}, {"L": 16, "T": 4.44, "U": 0.54},
              {"L": 16, "T": 4.60, "U": 0.20}, {"L": 32, "T": 4.52, "U": 0.40},
              {"L": 32, "T": 4.53, "U": None}]
    rows = bench.binder_table(binder)
    by = {(r["L"], r["T_lo"]): r for r in rows}
    assert by[(16, 4.40)]["n"] == 2 and abs(by[(16, 4.40)]["U"] - 0.52) < 1e-12
    assert abs(by[(16, 4.40)]["err"] - 0.02) < 1e-12     # std 0.0283 / sqrt(2)
    assert by[(16, 4.55)]["n"] == 1 and by[(16, 4.55)]["err"] is None  # T = 4.60 falls in the last bin
    assert by[(32, 4.50)]["n"] == 1                        # lattices without samples are left out
    assert (16, 4.45) not in by
