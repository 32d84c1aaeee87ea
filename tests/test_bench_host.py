"""Host logic of bench.py that needs no GPU: the code digest that decides whether
the committed ncu counters still describe the kernels, and the summaries it reads."""

import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def write(tmp_path, name, text):
    p = tmp_path / name
    p.write_text(text)
    return str(p)


def test_code_digest_ignores_comments_and_blank_lines(bench, tmp_path):
    a = write(tmp_path, "a.cu", "int f() {\n    return 1;  // one\n}\n")
    b = write(tmp_path, "b.cu", "// a header\nint f() {\n\n    return 1;\n}   \n")
    c = write(tmp_path, "c.cu", "int f() {\n    return 2;\n}\n")
    assert bench.source_digest(a) == bench.source_digest(b)
    assert bench.source_digest(a) != bench.source_digest(c)


def test_committed_summaries_parse(bench):
    for kind, (prof, src) in bench.PROFILES.items():
        text = open(os.path.join(ROOT, prof)).read()
        keys = [line.split(": ", 1)[0] for line in text.splitlines() if ": " in line]
        assert "dram_bytes_per_launch" in keys and "source_code_sha256_prefix" in keys, prof
        assert os.path.exists(os.path.join(ROOT, src))
    text = open(os.path.join(ROOT, "profiles/iteration_dram_ellipses1024.md")).read()
    assert "dram_bytes_per_iteration: " in text
    assert "source_code_sha256_prefix_conv: " in text
    assert "source_code_sha256_prefix_transform: " in text


def test_counters_are_withheld_when_the_kernel_code_changes(bench, tmp_path, monkeypatch):
    src = write(tmp_path, "k.cu", "__global__ void k() {}\n")
    prof = write(tmp_path, "k.md", "dram_bytes_per_launch: 1234\nsource_code_sha256_prefix: "
                 + bench.source_digest(src)[:16] + "\n")
    monkeypatch.setitem(bench.PROFILES, "stencil", (prof, src))
    assert bench.measured_traffic("stencil") == 1234
    open(src, "a").write("// a comment only\n")
    assert bench.measured_traffic("stencil") == 1234
    open(src, "a").write("__global__ void k2() {}\n")
    assert bench.measured_traffic("stencil") is None


def test_bench_stable_alpha_follows_the_pinned_symbol_ratio(bench):
    """The bench's per-PSF alpha (its own NumPy restatement of the stability ratio)
    equals the reading pinned on the oracle's symbols: for the bench's motion PSF
    0.3, for the 2048^2 workload's Gaussian 0.1, and for random batch PSFs the
    smallest half-decade value whose oracle ratio stays below 2."""
    import numpy as np

    import oracle as O
    from paper_1211_0393_gb300 import workloads as W
    assert bench.stable_alpha(W.psf_config2()) == 0.3
    assert bench.stable_alpha(W.psf_config4()) == 0.1

    def oracle_ratio(h, alpha):
        q1, q2 = O.psf_support(h)
        x = np.linspace(0, np.pi, 181)
        x1, x2 = x[:, None], x[None, :]
        hp = np.zeros((181, 181), dtype=complex)
        hm = np.zeros_like(hp)
        for a in range(-q1, q1 + 1):
            for b in range(-q2, q2 + 1):
                hp += h[a + q1, b + q2] * np.exp(-1j * (a * x1 + b * x2))
                hm += h[a + q1, b + q2] * np.exp(-1j * (-a * x1 + b * x2))
        e = np.maximum(np.abs(hp) ** 2, np.abs(hm) ** 2)
        return float((e / (O.symbol(O.symmetrize(h), x, x) ** 2 + alpha)).max())

    for sp in W.batch_specs(6):
        a = bench.stable_alpha(sp["psf"])
        assert a == 1.0 or oracle_ratio(sp["psf"], a) < 2.0
        smaller = [v for v in bench.ALPHA_GRID if v < a]
        if smaller:
            assert oracle_ratio(sp["psf"], smaller[-1]) >= 2.0
