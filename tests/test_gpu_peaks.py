"""The integer-pipe measurement kernels behind the sweep's roofline
(pa_measure_pipe_peak, pa_measure_rng_peak): they run, report a positive
rate, and stay below the issue limit of one warp instruction per clock per
SM sub-partition (4 x 32 lanes per SM per clock) -- a rate above it would
mean the compiler shortened the dependency chains."""
import pytest

pytestmark = pytest.mark.gpu


def _issue_limit_gops():
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return sms * 128 * 2.1  # lanes per ns at 2.1 GHz, above the 2.07 GHz maximum


@pytest.mark.parametrize("pipe", [0, 1, 2])
def test_pipe_peak_in_range(pipe):
    import paper_1703_03676_gb300 as pa
    v = pa.measure_pipe_peak(pipe, 2048)
    assert 0 < v < _issue_limit_gops()


def test_wide_multiply_slower_than_logic():
    """A 32x32->64 multiply occupies its pipe longer than a logic op: the
    premise of counting multiplies as the sweep's binding resource."""
    import paper_1703_03676_gb300 as pa
    assert pa.measure_pipe_peak(pa.PIPE_WIDE_MUL, 4096) < pa.measure_pipe_peak(pa.PIPE_LOP3, 4096)


def test_pipe_peak_rejects_bad_arguments():
    import paper_1703_03676_gb300 as pa
    with pytest.raises(RuntimeError):
        pa.measure_pipe_peak(3, 2048)
    with pytest.raises(RuntimeError):
        pa.measure_pipe_peak(0, 2)


def test_rng_peak_below_wide_multiply_bound():
    """Philox4x32-10 needs at least 17 lane-varying wide multiplies per 4
    words here, so its word rate is bounded by 4/17 of the multiply rate."""
    import paper_1703_03676_gb300 as pa
    words = pa.measure_rng_peak(2048)
    mul = pa.measure_pipe_peak(pa.PIPE_WIDE_MUL, 4096)
    assert 0 < words <= mul * 4.0 / 17.0 * 1.05
