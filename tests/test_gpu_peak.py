"""The FMA-throughput microbenchmark (dugks_alu_peak) that gives the FP64
form's roofline denominator: sane rates on GB300 and argument checks.

GB300 issues FP64 at a small fraction of its FP32 rate; the checks are loose
plausibility bounds (per SM per clock: FP64 at most 4 flops, FP32 at most
256), not performance targets."""
import pytest

import paper_1709_05458_gb300 as P

pytestmark = pytest.mark.gpu


def test_alu_peak_rates_are_plausible(cuda):
    torch = cuda
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    out = torch.zeros(sms * 4 * 256, dtype=torch.float64, device="cuda")
    rates = {}
    for name, kind, iters in (("fp64", P.ALU_FP64, 200), ("fp32", P.ALU_FP32, 4000),
                              ("fp32x2", P.ALU_FP32X2, 4000)):
        P.dugks_alu_peak(kind, iters, 4, out)            # warm-up
        fl, ms = P.dugks_alu_peak(kind, iters, 4, out)
        assert fl == 2 * 8 * 16 * iters * 256 * sms * 4 * (2 if kind == P.ALU_FP32X2 else 1)
        assert ms > 0
        rates[name] = fl / (ms * 1e-3)
        assert bool(torch.isfinite(out).all())
    ghz_max = 2.2
    assert 0.1e12 < rates["fp64"] <= sms * 4 * ghz_max * 1e9
    assert rates["fp32"] <= sms * 256 * ghz_max * 1e9
    assert rates["fp32"] > 10 * rates["fp64"]
    assert rates["fp32x2"] > 0.5 * rates["fp32"]


def test_alu_peak_rejects_short_buffer(cuda):
    torch = cuda
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(P.DugksError) as e:
        P.dugks_alu_peak(P.ALU_FP64, 10, 4, out)
    assert e.value.code == P.DUGKS_EINVAL
