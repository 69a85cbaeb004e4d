"""bs_fma_rate: the measured fma-chain rates are positive, finite and in the range of this part's pipes
(float32 near the nominal 152 SMs x 128 lanes x 2 x clock, packed float32x2 no faster per lane, float64 far
below float32)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0712_1695_gb300 as bs  # noqa: E402
from paper_0712_1695_gb300.binding import BS_ERR_ARG, BSError  # noqa: E402


def test_fma_rates():
    bs.build()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = n_sm * 128 * 2 * 2.07e9 / 1e12  # upper clock bound of the part
    f64, f32, f32x2 = (bs.bs_fma_rate(k) for k in (0, 1, 2))
    assert 0.2 * nominal < f32 <= 1.05 * nominal
    assert 0.2 * nominal < f32x2 <= 1.05 * nominal
    assert 0 < f64 < 0.5 * f32
    with pytest.raises(BSError) as ei:
        bs.bs_fma_rate(3)
    assert ei.value.code == BS_ERR_ARG
