"""bench.py's accounting (CPU only): the algorithmic byte and flop counts the
roofline figures divide by, and the source hash that ties stored DRAM
traffic to the kernel code it was measured on."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)


def test_lhat_bytes_at_1024():
    # volume read (4 B/voxel) + u1 written and read for the h/2 + 1 paired
    # planes (16 B per point) + d_hat written (8 B per point), per direction
    n = 1024
    one = 4 * n ** 3 + 16 * n * n * (n // 2 + 1) + 8 * n ** 3
    assert bench.lhat_bytes(n, n, n, n, n) == one
    assert 2 * one == 42983227392


def test_iteration_bytes_add_up():
    n, k = 64, 4
    K = D = n ** 3
    vox = sum(32 + (12 if i else 0) + 12 + 4 + 8 + (4 if i else 0) + (8 if i == k - 1 else 0) for i in range(k)) + 80
    assert vox == 280 + 80
    want = k * 2 * bench.lhat_bytes(n, n, n, n, n) + K * vox + D * k * 32
    assert bench.admm_iteration_bytes(n, n, n, n, n, k) == want


def test_spread_point_flops():
    # 64 cells x (complex accumulate of a real weight times a value) + 16 weights
    assert bench.spread_point_flops(4) == 64 * 4 + 16


def test_source_hash_ignores_comments_and_layout():
    a = "int f(int x) {\n  return x + 1;  // one more\n}\n"
    b = "/* header */\nint f(int x) {\n\n    return x + 1;\n}"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench._strip_comments(a) == bench._strip_comments(b)
    assert bench._strip_comments(a) != bench._strip_comments(c)
    assert len(bench.source_hash()) == 64
