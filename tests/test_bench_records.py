"""Host logic of the bench's counter records (profiles/traffic.txt): a DRAM-byte
or instruction count per particle is reported only while the kernel source
hashes to the value recorded beside it, so a number taken from an older kernel
is never attached to a newer one."""
import hashlib
import os
import shutil

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join("paper_1705_04368_gb300", "csrc", "mdlg_md.cu")


def _tree(tmp_path, record_sha, extra=""):
    (tmp_path / "paper_1705_04368_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, SRC), tmp_path / SRC)
    (tmp_path / "profiles" / "traffic.txt").write_text(
        f"kernel=k_step src_sha={record_sha} dram_bytes_per_particle=90.5 {extra}"
        "source=profiles/x.md\n")
    return tmp_path


def _sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def test_record_used_while_source_unchanged(tmp_path, monkeypatch):
    root = _tree(tmp_path, _sha(os.path.join(ROOT, SRC)), "warp_inst_per_particle=21.5 ")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic_record("k_step") == 90.5
    assert bench._traffic_record("k_step", "warp_inst_per_particle") == 21.5
    assert bench._traffic_record("k_nlist") is None


def test_record_dropped_after_a_source_change(tmp_path, monkeypatch):
    root = _tree(tmp_path, _sha(os.path.join(ROOT, SRC)))
    with open(root / SRC, "a") as f:
        f.write("\n// changed\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic_record("k_step") is None


def test_missing_key_or_file_gives_none(tmp_path, monkeypatch):
    root = _tree(tmp_path, _sha(os.path.join(ROOT, SRC)))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic_record("k_step", "warp_inst_per_particle") is None
    os.remove(root / "profiles" / "traffic.txt")
    assert bench._traffic_record("k_step") is None

