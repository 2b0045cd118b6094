"""Host logic of bench.py (no GPU): the byte models behind the roofline
fractions, and the digest gate that keeps a DRAM-traffic figure only while
the kernel's source is the one that was captured."""

import hashlib
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


DIM, NNZ = 172684, 102601752   # config 1


def test_spmm_bytes_model(bench):
    # CSR streamed once (4 B column + 4 B value per nonzero, 8 B row pointer
    # per row and one more), X read once (8 FP32 per row), Y written once
    csr = 8 * NNZ + 8 * (DIM + 1)
    assert bench.algorithmic_bytes("k_spmm", DIM, NNZ) == csr + 32 * DIM + 32 * DIM == 833247272
    # inside the solve Y is the FP64 Lanczos block
    assert bench.algorithmic_bytes("k_spmm", DIM, NNZ, y_bytes=8) == csr + 32 * DIM + 64 * DIM == 838773160
    assert bench.algorithmic_bytes("k_spmm16", DIM, NNZ) == csr + 64 * DIM + 64 * DIM


def test_fill_and_build_bytes_model(bench):
    assert bench.algorithmic_bytes("k_fill_rows", DIM, NNZ) == 8 * NNZ + 8 * (DIM + 1) == 822195496
    assert bench.algorithmic_bytes("build_H", DIM, NNZ) == 8 * NNZ + 12 * DIM + 8
    assert bench.algorithmic_bytes("k_count_rows", DIM, NNZ) is None


def test_traffic_kept_only_for_the_captured_source(bench, tmp_path, monkeypatch):
    src_a = tmp_path / "a.cu"
    src_b = tmp_path / "b.cu"
    src_a.write_text("kernel a\n")
    src_b.write_text("kernel b, edited after its capture\n")
    dig_a = hashlib.sha256(src_a.read_bytes()).hexdigest()[:16]
    traffic = tmp_path / "traffic.txt"
    traffic.write_text("# comment line k_x 1 a.cu %s\n"
                       "k_a 123000000 a.cu %s\n"
                       "k_b 456000000 b.cu %s\n"
                       "k_c 789000000 missing.cu %s\n" % (dig_a, dig_a, dig_a, dig_a))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(traffic))
    assert bench.ncu_traffic() == {"k_a": 123000000.0}


def test_committed_traffic_file_parses(bench):
    # every data line names an existing source file and carries a 16-digit digest
    with open(bench.TRAFFIC_FILE) as f:
        rows = [line.split() for line in f if line.strip() and not line.startswith("#")]
    assert rows
    for name, nbytes, src, digest in (r[:4] for r in rows):
        assert float(nbytes) > 0
        assert os.path.exists(os.path.join(ROOT, src)), src
        assert len(digest) == 16 and int(digest, 16) >= 0
