"""Host arithmetic of bench.py (CPU): the algorithmic byte model behind roofline.frac and the
rule that drops a stored DRAM-traffic record once the kernel source has changed."""
import json
import os

import numpy as np

import nmc_inputs as W


def test_byte_model_by_hand():
    import bench
    # clause 1: three literals (each occurrence sees 2 neighbours), clause 2: two (1 each)
    lits = np.array([[1, -2, 3, 0], [2, 4, 0, 0]], dtype=np.int32)
    # 33 replicas = 2 words; neighbour words 3*2 + 2*1 = 8, own word read + write 2 * 4 vars,
    # occurrence entries 5 x 4 int32, beta row 4 floats
    want = 8 * 2 * 4 + 2 * 4 * 2 * 4 + 5 * 4 * 4 + 4 * 4
    assert bench.algorithmic_bytes_per_sweep(lits, 4, 33) == want == 224
    # replica count enters only through whole 32-replica words
    assert bench.algorithmic_bytes_per_sweep(lits, 4, 64) == 224
    assert bench.algorithmic_bytes_per_sweep(lits, 4, 1) == 224 - (8 + 8) * 4


def test_byte_model_of_the_50k_bench_instance():
    """4-SAT, N = 50,000, alpha 9.6 (M = 480,000), 1,024 replicas (32 words):
    480,000 x 4 x 3 neighbour words x 32 x 4 B = 737.28 MB, own words 2 x 50,000 x 32 x 4 B =
    12.8 MB, occurrence entries 1,920,000 x 4 x 4 B = 30.72 MB, beta row 0.2 MB: 781 MB."""
    import bench
    n = 50_000
    lits = W.random_ksat(n, 9.6, 4, 2111)
    assert lits.shape == (480_000, 4) and np.all(lits != 0)
    assert bench.algorithmic_bytes_per_sweep(lits, n, 1024) == 781_000_000


def test_traffic_record_dropped_when_source_changes(tmp_path, monkeypatch):
    import bench
    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel v1")
    import hashlib
    h = hashlib.sha256(b"kernel v1").hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    rec = {"k": {"workload": "w", "source_sha256_16": h, "source": "k.cu",
                 "dram_bytes_read": 1000, "dram_bytes_write": 24}}
    (tmp_path / "profiles" / bench.TRAFFIC_FILE).write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.captured_traffic("k", "w") == 1024
    assert bench.captured_traffic("k", "other workload") is None
    assert bench.captured_traffic("missing", "w") is None
    src.write_bytes(b"kernel v2")
    assert bench.captured_traffic("k", "w") is None


def test_committed_traffic_record_names_an_existing_source():
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "profiles", bench.TRAFFIC_FILE)) as f:
        rec = json.load(f)
    for r in rec.values():
        assert os.path.exists(os.path.join(root, r["source"]))
        assert r["dram_bytes_read"] > 0 and r["dram_bytes_write"] >= 0
