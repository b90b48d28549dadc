"""Measurement and input aids on the GPU: the FMA-rate probe behind the
roofline's peak, and the device right-hand side."""
import numpy as np
import pytest
import torch

import paper_2507_17053_gb300 as G
import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_peak_probe_and_device_rhs():
    """The FMA-rate probe returns a rate near the GPU's FP64 / FP32 pipes
    (GB300: 2 / 128 lane-FMAs per SM per clock), and the device right-hand
    side equals the host one."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    p64, p32 = G.sbm_peak_probe(64), G.sbm_peak_probe(32)
    # clocks between 1.0 and 2.1 GHz
    assert 2 * sms * 1.0 <= p64 <= 2 * sms * 2.1, p64
    assert 128 * sms * 1.0 <= p32 <= 128 * sms * 2.1, p32
    P = G.Problem.from_workload(S.SPHERE_3D_Q4.resized(7, degree=2))
    bd = P.rhs_device(0)
    torch.cuda.synchronize()
    assert np.array_equal(bd.cpu().numpy(), P.rhs(0))
