"""Band-passed Ricker source wavelet — TEST INFRASTRUCTURE ONLY (the same
import rule as the rest of ``oracle/``: tests, smoke() and bench.py's CPU legs).

The paper defines the wavelet of its production runs (Sec. "Source Wavelet",
Tab. bands) by library calls, and this module writes that definition out with
the same routines as steps: a Ricker pulse of peak frequency f0 centred at
t0 = 1/f0; a 4th-order Butterworth band-pass at the band corners designed as
second-order sections (scipy.signal.butter) and applied forward and backward
(scipy.signal.sosfiltfilt, zero phase); division by the l2 norm; scaling by
sqrt(B / 24 Hz), B = f_hi - f_lo. Reading R9: "4th-order" is the order
argument of the band-pass design (8 poles).

Pins (tests/test_oracle_pins.py): the Ricker's amplitude spectrum peaks at f0
(closed form f^2 exp(-f^2/f0^2)); the l2 norm equals sqrt(B / 24 Hz); the
forward-backward gain for a pure tone equals the squared analog Butterworth
magnitude 1 / (1 + ((W^2 - W0^2) / (W B_W))^(2N)) at the prewarped frequency
W = 2 fs tan(pi f / fs) (bilinear transform); a pulse centred in the record
comes out symmetric (zero phase).
"""
import math

import numpy as np

# (f_lo, f_hi, f0) of the five bands (Tab. bands; f0 from Sec. "Source Wavelet")
BANDS = [(3.0, 6.0, 4.50), (3.0, 8.5, 5.75), (3.0, 12.0, 7.50), (3.0, 17.5, 10.25), (3.0, 25.0, 14.00)]


def ricker(f0, t0, dt, nt):
    """(1 - 2 (pi f0 tau)^2) exp(-(pi f0 tau)^2), tau = n dt - t0, in FP64."""
    tau = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def bandpass(x, f_lo, f_hi, dt, order=4):
    """Zero-phase Butterworth band-pass of a record (design, then forward-backward)."""
    from scipy import signal
    sos = signal.butter(order, [f_lo, f_hi], btype="bandpass", fs=1.0 / dt, output="sos")
    return signal.sosfiltfilt(sos, x)


def bandpass_ricker(f0, f_lo, f_hi, dt, nt, order=4):
    """The production source wavelet, FP64 [nt]."""
    w = bandpass(ricker(f0, 1.0 / f0, dt, nt), f_lo, f_hi, dt, order)
    return w / np.linalg.norm(w) * math.sqrt((f_hi - f_lo) / 24.0)
