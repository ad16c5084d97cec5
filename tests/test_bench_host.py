"""Host logic of bench.py, without a GPU: the roofline's choice of bound and its fractions,
the source hash that ties a committed DRAM capture to a kernel's definition, the operand
roundings behind the accuracy statistics (against torch's own BF16 and E4M3 conversions),
and the job-value arithmetic."""
import os
import tempfile

import numpy as np
import pytest

import bench

PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}


def _stages(gemm_ms, nsub):
    stage_ms = [0.0] * 8
    stage_ms[2] = gemm_ms * 1.5          # the user stage holds more than the GEMM kernel
    stage_ms[6] = gemm_ms                # the GEMM kernel alone
    launches = [nsub] + [0] * 7
    return stage_ms, launches


def test_user_pass_bound_follows_its_arithmetic_intensity():
    d = dp = 128
    stage_ms, launches = _stages(0.3, 2)
    # few scores per user row streamed: under the ridge, so the bound is HBM
    st = {"tc_scores": 1_000_000, "tc_rows": 2_000_000}
    r = bench.stage_rooflines(stage_ms, launches, st, d, dp, PEAKS, "measured")["user_pass"]
    by = (2 * dp + 12) * 2_000_000
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(by / 0.3e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["hbm_gbs"])
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(by / 2)
    assert r["launch_ms"] == pytest.approx(0.15)
    assert r["ridge"] == pytest.approx(1900e12 / 6800e9)
    assert r["other_bound"]["bound"] == "tensor"
    assert r["other_bound"]["frac"] == pytest.approx(2 * d * 1e6 / 0.3e-3 / 1e12 / PEAKS["bf16_tflops"])
    # many scores per row: over the ridge, so the bound is the tensor pipe
    st = {"tc_scores": 10_000_000_000, "tc_rows": 2_000_000}
    r = bench.stage_rooflines(stage_ms, launches, st, d, dp, PEAKS, "measured")["user_pass"]
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(2 * d * 1e10 / 0.3e-3 / 1e12)
    assert r["arithmetic_intensity"] > r["ridge"]


def test_other_stage_rooflines_and_the_dominant_stage():
    stage_ms = [0.01, 0.1, 0.5, 0.2, 0.05, 0.0, 0.3, 0.15]
    launches = [1] + [0] * 7
    st = {"tc_scores": 1_000_000, "tc_rows": 2_000_000, "block_col_pairs": 5_000_000, "items_scanned": 10 ** 9}
    roofs = bench.stage_rooflines(stage_ms, launches, st, 128, 128, PEAKS, "measured")
    fp32_peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert roofs["block_pass"]["bound"] == "alu"
    assert roofs["block_pass"]["peak"] == pytest.approx(fp32_peak)
    assert roofs["block_pass"]["achieved"] == pytest.approx(2 * 128 * 5e6 / 0.1e-3 / 1e12)
    assert roofs["kmips_decision"]["achieved"] == pytest.approx(2 * 128 * 1e9 / 0.15e-3 / 1e12)
    name, roof = bench.dominant(stage_ms, roofs)
    assert name == "user_pass" and roof is roofs["user_pass"]
    # no counters, no roofline
    assert bench.stage_rooflines(stage_ms, launches, {}, 128, 128, PEAKS, "measured") == {}


def test_kernel_source_hash_covers_the_definition_only():
    src = """// foo_kernel( is named in this comment
template <int A>
__global__ void foo_kernel(int x) {
  if (x) {
    x += A;
  }
}

__global__ void bar_kernel(int y) { y += 1; }

void launch() { foo_kernel<1><<<1, 1>>>(0); }
"""
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "k.cu")

        def h(text, kernel="foo_kernel"):
            with open(p, "w") as f:
                f.write(text)
            return bench.kernel_source_hash(p, kernel)

        base = h(src)
        assert base is not None and len(base) == 16
        assert h(src) == base                                                  # deterministic
        assert h(src.replace("y += 1", "y += 2")) == base                      # another kernel
        assert h(src.replace("void launch() {", "void launch2() {")) == base   # a launch site
        assert h(src.replace("x += A;", "x += 2 * A;")) != base                # its body
        assert h(src.replace("template <int A>", "template <int B>")) != base  # its template line
        assert h(src, "baz_kernel") is None


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    # exact ties: the low 16 bits 0x8000, with both parities of the kept part
    b = x.view(np.uint32).copy()
    b[:2000] = (b[:2000] & np.uint32(0xFFFF0000)) | np.uint32(0x8000)
    x = b.view(np.float32)
    got = bench._bf16_round(x)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_e4m3_rows_match_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn in this torch")
    rng = np.random.default_rng(1)
    X = (rng.standard_normal((64, 100)) * np.exp(rng.uniform(-8, 8, (64, 1)))).astype(np.float32)
    X[3] = 0.0                                          # a zero row: scale 0, all codes 0
    X[5, :50] *= 1e-6                                   # subnormal codes in one row
    y8, scale = bench._e4m3_rows(X)
    mx = np.abs(X).max(axis=1)
    inv = np.where(mx > 0, np.float32(448.0) / np.where(mx > 0, mx, 1), 0).astype(np.float32)
    scaled = (X * inv[:, None]).astype(np.float32)
    want = torch.from_numpy(scaled).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(y8, want)
    assert np.allclose(scale, mx.astype(np.float64) / 448.0, rtol=1e-7)
    assert np.all(np.abs(y8) <= 448.0) and np.all(y8[3] == 0)


def test_whole_job_value_and_f1():
    value, t_ms = bench.whole_job_value(1000.0, 10000, 400, 2, lambda x: x)
    assert t_ms == 1000.0 and value == pytest.approx(10000 * 400 * 2 / 1.0)
    value, t_ms = bench.whole_job_value(500.0, 100, 10, 4, lambda x: 2 * x)   # the slowest rank's time
    assert t_ms == 1000.0 and value == pytest.approx(100 * 10 * 4 / 1.0)
    assert bench.f1_sets([1, 2], [2, 3]) == pytest.approx(0.5)
    assert bench.f1_sets([], []) == 1.0
    assert bench.f1_sets([1], []) == 0.0
