"""Host logic of bench.py, on the CPU:
- the algorithmic bytes per node update, re-derived from array counts;
- the ncu traffic records, which are used only when they were taken on the
  kernel source as it is, and the committed records, which match it."""
import os

import pytest

import bench


def test_bytes_per_node_from_array_counts():
    # D2Q9: f and g (9 arrays each) read and written once, S read and written,
    # FP32 also the rest population's low word (one more f array)
    assert bench.BYTES_PER_NODE["fp32"] == (9 + 1 + 9) * 4 * 2 + 2 * 4
    assert bench.BYTES_PER_NODE["fp64"] == (9 + 9) * 8 * 2 + 2 * 8
    # D3Q19 likewise; 16-bit offsets: 2 x 19 u16 read and written, six FP32
    # macros read and written, S read and written
    assert bench.BYTES_PER_NODE_3D["fp32"] == (19 + 1 + 19) * 4 * 2 + 2 * 4
    assert bench.BYTES_PER_NODE_3D["fp64"] == (19 + 19) * 8 * 2 + 2 * 8
    assert bench.BYTES_PER_NODE_3D["f16off"] == (19 + 19) * 2 * 2 + 6 * 4 * 2 + 2 * 4
    assert bench.BYTES_PER_NODE_3D["bf16off"] == bench.BYTES_PER_NODE_3D["f16off"]


@pytest.mark.parametrize("esz,lo", [(4, 1), (8, 0)])
def test_adjoint_bytes_per_node_from_array_counts(esz, lo):
    step = ((9 + 9 + lo) * 2 + 2) * esz            # recorded forward step
    recompute = step + 5 * esz                      # + phi, mu, p, ux, uy written
    # adj_local reads f, g (+ lo) at the pulled sources, the five moments,
    # lambda_f (9) + lambda_phi (1), lambda_g (9), lambda_S; writes lambda_f,
    # lambda_g, lambda_S, lambda_phi, lambda_mu, lambda_grad_phi (2) and
    # lambda_grad_mu (2)
    local = (9 + 9 + lo + 5 + 10 + 9 + 1) * esz + (9 + 9 + 1 + 1 + 1 + 2 + 2) * esz
    # adj_mu_phi reads lambda_mu, lambda_grad_mu (2), phi, lambda_phi,
    # lambda_grad_phi (2); writes lambda_phi_tot
    mu_phi = (1 + 2 + 1 + 1 + 2) * esz + esz
    assert bench.adjoint_bytes_per_node(esz) == step + recompute + local + mu_phi


def test_traffic_record_needs_the_current_kernel_source(tmp_path, monkeypatch):
    rec = tmp_path / "t.txt"
    rec.write_text("# comment: 1\nkernel_sha: %s\ndram_bytes_per_step: 1234\n" % bench.kernel_hash())
    monkeypatch.setitem(bench.TRAFFIC_FILES, "per_step", str(rec))
    assert bench.ncu_traffic("per_step") == 1234.0
    rec.write_text("kernel_sha: 0000000000000000\ndram_bytes_per_step: 1234\n")
    assert bench.ncu_traffic("per_step") is None
    monkeypatch.setitem(bench.TRAFFIC_FILES, "per_step", str(tmp_path / "missing.txt"))
    assert bench.ncu_traffic("per_step") is None


def test_committed_traffic_records_match_the_kernel_source():
    """A kernel change must come with a new ncu capture (else the bench
    reports traffic as null): the committed records carry the source hash."""
    for mode, path in bench.TRAFFIC_FILES.items():
        assert os.path.exists(path), path
        assert bench.ncu_traffic(mode) is not None, (mode, "re-capture the DRAM traffic")
        # the recorded bytes are close to the algorithmic 2 x 1024^2 x 160 B per step
        assert 0.8 < bench.ncu_traffic(mode) / (2 * 1024 * 1024 * 160) < 1.05


def test_kernel_hash_follows_code_not_comments(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", ("k.cu",))
    src.write_text("// a step\nint f(int x) { return x + 1; }  // plus one\n")
    h = bench.kernel_hash()
    src.write_text("/* the step,\n   reworded */\n\nint f(int x) { return x + 1; }\n")
    assert bench.kernel_hash() == h
    src.write_text("// a step\nint f(int x) { return x + 2; }  // plus one\n")
    assert bench.kernel_hash() != h
