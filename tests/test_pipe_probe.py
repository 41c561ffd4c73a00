"""The pipe probe behind the bench's ALU rooflines: it compiles for sm_103a (CPU), and on the GPU
its packed f32x2 FMA rounds every half exactly like the scalar FMA, its rates are positive, and
the RK4 arithmetic on register-resident sites runs no faster than the pipe it issues to."""
import pytest

import pipe_probe


def test_probe_compiles():
    exe = pipe_probe.compile_probe()
    assert exe.endswith("pipe_probe")


@pytest.mark.gpu
def test_probe_rates_and_packed_bit_identity():
    r = pipe_probe.run()
    assert r["packed_vs_scalar_fma_mismatches"] == 0 and r["packed_bit_check_values"] > 0
    for key in ("dfma_per_s", "dadd_per_s", "ffma_scalar_16chains_per_s", "ffma_packed_16lanes_per_s", "copy_gbs",
                "rk4_fp64_regs_inst_per_s", "rk4_fp32k_regs_lane_ops_per_s", "rk4_fp64_regs_smem_roundtrip_inst_per_s"):
        assert r[key] > 0, key
    # every FP64 instruction of the step can issue as a DFMA: the stream cannot beat that rate
    assert r["rk4_fp64_regs_inst_per_s"] <= 1.02 * r["dfma_per_s"]
    assert r["rk4_fp32k_regs_lane_ops_per_s"] <= 1.02 * max(r["ffma_packed_16lanes_per_s"],
                                                              r["ffma_scalar_16chains_per_s"])
