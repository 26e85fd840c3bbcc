"""FP64 FMA rate of the device (the roof of the FP64 forms): plausible, stable,
and its argument checks."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_00641_gb300 import vlbm
    vlbm.load()
    return vlbm


def test_fp64_rate_is_plausible_and_stable(V):
    r1 = V.vlbm_measure_fp64_rate(4096)
    r2 = V.vlbm_measure_fp64_rate(8192)
    # a GB300's FP64 pipe is rated about 1.25 TFLOP/s: an FMA chain the compiler removed
    # would read far above, a serialised one far below
    assert 0.3 < r1 < 5.0, r1
    # twice the chain length: the same rate (the launch overhead is a small share)
    assert abs(r2 - r1) < 0.1 * r1, (r1, r2)


@pytest.mark.parametrize("iters", [0, -1, (1 << 20) + 1])
def test_fp64_rate_refuses_bad_arguments(V, iters):
    with pytest.raises(V.VlbmError) as e:
        V.vlbm_measure_fp64_rate(iters)
    assert e.value.status == V.VLBM_ERR_ARG
