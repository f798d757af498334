"""GPU parity of the post-processing (batched inverse FFT + blend, Section III.B with
Eq. (1)) and of its adjoint against the FP64 oracle, on seeded random spectra."""
import numpy as np
import pytest
import torch

import scenegen as sg
from helpers import np_, rel_l2

pytestmark = pytest.mark.gpu
TOL_SYNTH = {"fp64": 1e-12, "split": 1e-5}   # FFT rounding only: no index decisions here


@pytest.fixture(scope="module")
def rsim():
    import paper_2408_11472_gb300 as m
    return m


CASES = [
    # (n_gates, n_doppler, n_fast, pulse0, n_pulses)
    (128, 64, 64, 0, 4096),      # cfg1 shape
    (128, 64, 64, 37, 300),      # ragged start and end
    (33, 16, 48, 5, 200),        # N_d < n_fast, odd gate count
    (20, 128, 64, 64, 129),      # N_d > n_fast, range ending on an update pulse
    (3, 1024, 100, 250, 333),    # largest transform
    (1, 2, 1, 0, 17),            # smallest transform, n_fast = 1
    (7, 4, 1023, 1, 2100),       # largest n_fast whose window the kernel tabulates
    (5, 64, 1024, 700, 2500),    # n_fast past the table: window evaluated per pulse
]
CDT = {"fp64": torch.complex128, "split": torch.complex64}


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("window", ["sqrt_linear", "sqrt_raised_cosine", "linear"])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_synth_parity(rsim, orc, case, window, precision):
    G, K, nf, p0, P = case
    rd = sg.RadarParams(n_gates=G)
    u0, S = rsim.spectra_range(p0, P, nf)
    T = sg.random_spectra(S, G, K, seed=G * 7 + K)
    Td = torch.as_tensor(T).to("cuda", CDT[precision])
    Y = np_(rsim.synth_pulses(rd, Td, u0, nf, p0, P, window))
    Yref = orc.synth(np_(Td).astype(np.complex128), u0, nf, p0, P, window)
    assert rel_l2(Y, Yref) <= TOL_SYNTH[precision]


@pytest.mark.parametrize("case", CASES[1:])
@pytest.mark.parametrize("window", ["sqrt_linear", "sqrt_raised_cosine"])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_synth_backward_parity(rsim, orc, case, window, precision):
    G, K, nf, p0, P = case
    rd = sg.RadarParams(n_gates=G)
    u0, S = rsim.spectra_range(p0, P, nf)
    GY = sg.random_iq(P, G, seed=P + G)
    GYd = torch.as_tensor(GY).to("cuda", CDT[precision])
    GT = np_(rsim.synth_pulses_backward(rd, GYd, S, u0, nf, K, p0, window))
    GTref = orc.synth_grad(np_(GYd).astype(np.complex128), S, u0, nf, K, p0, window)
    assert rel_l2(GT, GTref) <= TOL_SYNTH[precision]


def test_synth_adjoint_identity_on_gpu(rsim):
    """<G_Y, synth(T)> = <synth_backward(G_Y), T> in FP64 on the device."""
    rd = sg.RadarParams(n_gates=24)
    u0, S = rsim.spectra_range(10, 250, 40)
    T = torch.as_tensor(sg.random_spectra(S, 24, 32, 5)).cuda()
    GY = torch.as_tensor(sg.random_iq(250, 24, 6)).cuda()
    Y = rsim.synth_pulses(rd, T, u0, 40, 10, 250, "sqrt_linear")
    GT = rsim.synth_pulses_backward(rd, GY, S, u0, 40, 32, 10, "sqrt_linear")
    lhs = torch.vdot(GY.flatten(), Y.flatten()).real.item()
    rhs = torch.vdot(GT.flatten(), T.flatten()).real.item()
    assert lhs == pytest.approx(rhs, rel=1e-12)
