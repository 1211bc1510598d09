"""Host logic of bench.py, on the CPU:
- the algorithmic bytes per node update, re-derived from array counts;
- the ncu traffic records, which are used only when they were taken on the
  kernel source as it is, and the committed records, which match it."""
import os

import pytest

import bench


def test_bytes_per_node_from_array_counts():
    # algorithmic bytes of a node update: f and g (9 arrays each) read once and
    # written once, S read and written; the FP32 rest population's low word
    # is overhead (it shows in the measured traffic), not algorithmic
    assert bench.BYTES_PER_NODE["fp32"] == 152
    assert bench.BYTES_PER_NODE["fp32"] == (9 + 9) * 4 * 2 + 2 * 4
    assert bench.BYTES_PER_NODE["fp64"] == (9 + 9) * 8 * 2 + 2 * 8
    # D3Q19 likewise; 16-bit offsets: 2 x 19 u16 read and written, six FP32
    # macros read and written, S read and written
    assert bench.BYTES_PER_NODE_3D["fp32"] == (19 + 19) * 4 * 2 + 2 * 4 == 312
    assert bench.BYTES_PER_NODE_3D["fp64"] == (19 + 19) * 8 * 2 + 2 * 8
    assert bench.BYTES_PER_NODE_3D["f16off"] == (19 + 19) * 2 * 2 + 6 * 4 * 2 + 2 * 4 == 208
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
        # the recorded bytes are close to the algorithmic 2 x 1024^2 x 152 B per
        # step: plus the rest population's low word (8 B, 1.05x) and the halo
        # rows and columns that neighbouring tiles both read, when L2 does not
        # serve them (1.07x to 1.16x measured for the staged multi-step
        # kernel at 64 x 16 tiles); far above that would mean wasted re-reads
        assert 0.8 < bench.ncu_traffic(mode) / (2 * 1024 * 1024 * 152) < 1.2


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


def test_diag_cadence_puts_one_diagnostics_step_in_every_timed_region():
    class A:
        pass
    for steps, every in ((20, 100), (20, 20), (300, 100), (7, 3)):
        a = A()
        a.steps, a.diag_every = steps, every
        de = bench.diag_cadence(a)
        for t0 in range(0, 50):
            n = sum(1 for t in range(t0, t0 + steps) if t % de == 0)
            assert n >= 1
            assert n == -(-steps // de) or n == steps // de


@pytest.mark.parametrize("t0,k,de", [(5, 20, 20), (0, 20, 20), (5, 2000, 100), (3, 7, 3),
                                     (0, 1, 1), (17, 40, 100), (0, 2000, 5000), (7, 3000, 1500)])
def test_multi_step_launch_count_holds_one_diagnostics_step_each(t0, k, de):
    """Re-derive the launch split by brute force: walk the steps, start a new
    launch whenever the current one already holds a diagnostics step and the
    next step carries another, or already holds STEP_CAP (1024) steps."""
    launches, has_diag, n = 1, False, 0
    for t in range(t0, t0 + k):
        if n == 1024 or (t % de == 0 and has_diag):
            launches += 1
            has_diag, n = False, 0
        if t % de == 0:
            has_diag = True
        n += 1
    assert bench.STEP_CAP == 1024
    assert bench.launches_multi_step(t0, k, de) == launches


def test_partition_covers_every_case_once_and_balances_nodes():
    sizes = [n * n for n in (512, 64, 300, 301, 90, 512, 128, 77, 250, 400)]
    for world in (1, 2, 3, 4, 16):
        parts = bench.partition_cases(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        # greedy largest-first: no rank exceeds the mean by more than the largest case
        assert max(loads) - sum(sizes) / world <= max(sizes)
    assert bench.partition_cases(sizes, 1) == [list(range(len(sizes)))]
