"""Measured FMA rates (sph_fma_rate), the arithmetic roofline of PI.

GB300: 152 SMs x 128 float32 lanes x 2 FLOP at up to 2.07 GHz is 80.5 TFLOP/s;
the float64 rate is a small fraction of it.  The bands below are wide (clock
states vary); they catch a kernel that does not run or is optimised away."""
import pytest

from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def test_fma_rates_are_plausible():
    torch = need_gpu()
    from paper_1110_3711_gb300 import sph
    scratch = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    f32 = sph.sph_fma_rate("fp32", scratch, st)
    f64 = sph.sph_fma_rate("fp64", scratch, st)
    props = torch.cuda.get_device_properties(0)
    ceiling = props.multi_processor_count * 128 * 2 * 2.2e9
    assert 0.25 * ceiling < f32 < 1.05 * ceiling
    assert 0.0 < f64 < 0.5 * f32
    assert float(scratch.abs().sum()) == 0.0   # the guarded store never ran
