"""The benchmark's multiply-add probe (libnf_probe.so): flop count and values."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("packed,chains", [(0, 8), (1, 16), (2, 8)])
def test_probe_values_and_flop_count(packed, chains):
    import torch
    from paper_2110_11392_gb300 import probe
    n = probe.sink_floats()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert n == sms * 4 * 256
    sink = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    iters = 2048
    flop = probe.fma_probe(sink, iters, packed)
    torch.cuda.synchronize()
    # n threads x iters x 16 trips x 8 chains x (2 lanes if packed) x 2 flop
    assert flop == n * iters * 16 * 8 * (2 if packed == 1 else 1) * 2
    # x -> 0.999 x + 0.001 has its fixed point at 1: after 32768 trips every chain is 1
    assert torch.allclose(sink, torch.full_like(sink, float(chains)), rtol=0, atol=1e-3)


def test_probe_rejects_bad_arguments():
    import torch
    from paper_2110_11392_gb300 import probe
    small = torch.empty(8, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        probe.fma_probe(small, 16, True)
    sink = torch.empty(probe.sink_floats(), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        probe.fma_probe(sink, 0, True)
    with pytest.raises(ValueError):
        probe.fma_probe(sink, 16, 3)
