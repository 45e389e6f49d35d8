"""The arithmetic pipe probe (ssmul_debug_pipe_rate): every rate is positive
and within reach of the device's nominal peak (SMs x 2 binary64 or 128
binary32 operations per clock at the 2.07 GHz maximum clock)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1006_0405_gb300 import abi  # noqa: E402


def test_pipe_probe_rates_are_plausible():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for i, name in enumerate(abi.PIPE_OPS):
        s, g = abi.ssmul_debug_pipe_rate(i)
        assert s == abi.SSMUL_OK, name
        nominal = sms * (128 if name.startswith("f32") else 2) * 2.07
        assert 0.1 * nominal < g < 1.5 * nominal, (name, g, nominal)
    assert abi.ssmul_debug_pipe_rate(7)[0] == abi.SSMUL_INVALID_ARG
