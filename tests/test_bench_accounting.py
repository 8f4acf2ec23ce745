"""The benchmark's kernel accounting (bench.kernel_rooflines) on fabricated per-solve records:
the roofline object is the filter step kernel, its achieved rate is the executed slice work
(6 products x 8 n^2 flops per column-step) over the recorded device time, the fraction is
taken against the sustained BF16 peak, and the family with the most device time is named.
CPU only: no library call."""
import types

import pytest

import bench


def info(**kw):
    base = dict(ms_filter_lowp=0.0, ms_stage=[0.0] * 8, filter_col_steps=0, filter_col_steps_lowp=0,
                ms_filter_steps=0.0, filter_step_cols=0, ms_gemm_tc=0.0, gemm_tc_flop=0.0, ms_eig=0.0,
                eig_flop=0.0, ms_chol=0.0, chol_flop=0.0, eig_refined=0, eig_refine_iters=0,
                eig_f32_sweeps=0, eig_fallbacks=0, eig_sweeps=0, eig_rounds=0)
    base.update(kw)
    return types.SimpleNamespace(**base)


def test_filter_roofline_arithmetic():
    n = 2000
    # 1000 column-steps in 2 ms of step kernels; 1e12 algorithmic GEMM flops in 10 ms
    recs = [(0, info(ms_filter_steps=2.0, filter_step_cols=1000, ms_gemm_tc=10.0, gemm_tc_flop=1e12,
                     ms_filter_lowp=2.5, ms_stage=[0, 0, 2.5, 0, 0, 0, 0, 0],
                     filter_col_steps=1000, filter_col_steps_lowp=1000))]
    k, roof = bench.kernel_rooflines(recs, n, 1.05)
    pk, _ = bench.peaks()
    expect = 6 * 8.0 * n * n * 1000 / 2e-3 / 1e12
    assert roof["kernel"] == "tc_filter_step_kernel"
    assert roof["achieved"] == pytest.approx(expect)
    assert roof["frac"] == pytest.approx(expect / pk["bf16_tflops_sustained"])
    assert k["tc_filter_step_kernel"]["algorithmic_tflops"] == pytest.approx(expect / 6)
    # the digit GEMM: 78 executed products per algorithmic flop
    assert k["ozaki_kernel"]["achieved"] == pytest.approx(78 * 1e12 / 10e-3 / 1e12)
    assert roof["dominant_by_time"] == "ozaki_kernel"


def test_fp64_filter_family_only_with_fp64_column_steps():
    n = 500
    recs = [(0, info(ms_stage=[0, 0, 4.0, 0, 0, 0, 0, 0], filter_col_steps=300, filter_col_steps_lowp=100,
                     ms_filter_lowp=1.0))]
    k, roof = bench.kernel_rooflines(recs, n, 1.0)
    # 200 FP64 column-steps in the 3 ms not spent in the low-precision filter
    assert k["zgemm_kernel"]["achieved"] == pytest.approx(8.0 * n * n * 200 / 3e-3 / 1e12)
    assert roof["kernel"] == "zgemm_kernel"
