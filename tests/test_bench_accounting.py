"""bench.py's accounting (CPU only): the algorithmic byte and flop counts the
roofline figures divide by, and the source hash that ties stored DRAM
traffic to the kernel code it was measured on."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)


def test_lhat_bytes_at_1024():
    # the stage-boundary tensors of one L-hat at 1024^3, by their array sizes:
    # the volume read, the h/2 + 1 paired kv planes of u1 written by the z
    # stage and read by the plane stage, and d_hat written
    n = 1024
    vol = np.empty((n, n, n), dtype=np.float32).nbytes
    u1_plane = np.empty((n, n), dtype=np.complex64).nbytes
    dhat = np.empty((n, n, n), dtype=np.complex64).nbytes
    assert bench.lhat_bytes(n, n, n, n, n) == vol + 2 * (n // 2 + 1) * u1_plane + dhat
    assert 2 * bench.lhat_bytes(n, n, n, n, n) == 42983227392


# Each elementwise kernel of one Algorithm 2 outer iteration, with the arrays it
# reads and writes (volume arrays: bytes per voxel; data arrays: bytes per
# data point).  A stencil neighbour counts once.  Derived kernel by kernel from
# the launch sequence of admm_step, not from bench.py's formula.
def _kernel_table(n_inner):
    V, D = [], []
    for i in range(n_inner):
        first, last = i == 0, i == n_inner - 1
        # k_lsp_G: reads Gd, e[3], lambda[3]; from the 2nd step du, p, G_prev; writes G
        V.append(4 + 12 + 12 + (0 if first else 12) + 4)
        V.append(4 + 4 + 4)            # k_lsp_p: reads G, p, writes p
        V.append(4)                    # k_gradnorm2: reads p
        D.append(8)                    # k_cnorm2: reads L-hat p
        # k_axpy_u: reads p (+ du from the 2nd step), writes du; on the last step u read + written
        V.append(4 + (0 if first else 4) + 4 + (8 if last else 0))
        D.append(24)                   # k_axpy_r: reads r, L-hat p, writes r (compensation not counted)
    V.append(4 + 4 + 12 + 12 + 12 + 12 + 12)  # k_rsp: reads u, du, e, lambda; writes e, lambda, dpsi
    V.append(12)                       # k_divnorm2: reads dpsi
    return sum(V), sum(D)


def test_iteration_bytes_match_the_kernel_table():
    n, k = 64, 4
    vox, dat = _kernel_table(k)
    want = k * 2 * bench.lhat_bytes(n, n, n, n, n) + n ** 3 * vox + n ** 3 * dat
    assert bench.admm_iteration_bytes(n, n, n, n, n, k) == want


def test_spread_point_flops():
    # one point: its 8 x 8 cells, each a complex accumulation of a real weight
    # times the value (2 multiply-adds = 4 flops), plus its 16 separable weights
    cells = np.ones((8, 8))
    assert bench.spread_point_flops(4) == int(cells.sum()) * 4 + 2 * 8


def test_source_hash_ignores_comments_and_layout():
    a = "int f(int x) {\n  return x + 1;  // one more\n}\n"
    b = "/* header */\nint f(int x) {\n\n    return x + 1;\n}"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench._strip_comments(a) == bench._strip_comments(b)
    assert bench._strip_comments(a) != bench._strip_comments(c)
    assert len(bench.source_hash()) == 64
