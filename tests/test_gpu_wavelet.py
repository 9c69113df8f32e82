"""GPU band-passed Ricker wavelet (sim_wavelet_bandpass) against the oracle's
definition (scipy design + forward-backward filtering), for the paper's five
bands. The GPU designs the filter from the Butterworth definition itself and
filters in FP64: agreement to 1e-9 of the peak (the two factorise the filter
into sections differently, so only rounding differs); FP32 output to 1e-6."""
import numpy as np
import pytest

from oracle import wavelet as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_30541_gb300 as p
    p.abi.load()
    return p


@pytest.mark.parametrize("band", range(5))
def test_bands_match_oracle(pkg, band):
    lo, hi, f0 = W.BANDS[band]
    dt, nt = 1e-3, 8001
    ref = W.bandpass_ricker(f0, lo, hi, dt, nt)
    peak = np.abs(ref).max()
    g64 = pkg.bandpass_ricker(nt, dt, f0, lo, hi, dtype="float64").cpu().numpy()
    assert np.max(np.abs(g64 - ref)) <= 1e-9 * peak
    g32 = pkg.bandpass_ricker(nt, dt, f0, lo, hi, dtype="float32").cpu().numpy()
    assert np.max(np.abs(g32 - ref)) <= 1e-6 * peak
    host = np.zeros(nt, np.float64)  # host output through the same entry point
    pkg.sim_wavelet_bandpass(nt, dt, f0, lo, hi, 4, pkg.SIM_FP64, host)
    assert np.array_equal(host, g64)


def test_short_record_and_argument_errors(pkg):
    # the shortest record the definition accepts (one sample past the 27-sample reflection)
    ref = W.bandpass_ricker(10.25, 3.0, 17.5, 2e-3, 28)
    g = pkg.bandpass_ricker(28, 2e-3, 10.25, 3.0, 17.5, dtype="float64").cpu().numpy()
    assert np.max(np.abs(g - ref)) <= 1e-9 * np.abs(ref).max()
    for args in [(27, 2e-3, 10.25, 3.0, 17.5), (1, 1e-3, 5.0, 3.0, 6.0), (100, 1e-3, 5.0, 6.0, 3.0),
                 (100, 1e-3, 5.0, 3.0, 600.0)]:
        with pytest.raises(pkg.SimError):
            pkg.bandpass_ricker(*args)
