"""Pins of the oracle's Strouhal estimator (Sec. 4.2.1: St = L f / u_inf with
f the dominant frequency of the probe signal): known sinusoids, and the
refined peak against a direct scan of the windowed DFT on a fine grid."""
import math

import numpy as np

from oracle import strouhal as ost
from paper_0705_4371_gb300 import inputs


def test_recovers_known_frequencies():
    t = np.arange(50000)
    for f0 in (0.0012, 0.00287, 0.0131):
        sig = 0.05 + 0.01 * np.sin(2 * math.pi * f0 * t + 1.1) + 1e-3 * inputs.uniform(9, (t.size,))
        assert abs(ost.peak_frequency(sig) / f0 - 1.0) < 1e-4


def test_peak_matches_a_direct_scan_of_the_windowed_dft():
    # a two-tone signal: the estimate sits at the maximum of |sum w_n x_n
    # e^{-2 pi i f n}| found by scanning f directly (no FFT, no interpolation)
    n = 6000
    t = np.arange(n)
    x = np.sin(2 * math.pi * 0.01237 * t) + 0.3 * np.sin(2 * math.pi * 0.031 * t + 0.4)
    f_est = ost.peak_frequency(x)
    w = 0.5 - 0.5 * np.cos(2 * math.pi * t / (n - 1))
    y = (x - x.mean()) * w
    fs = np.linspace(0.0120, 0.0127, 1401)
    mag = np.abs(np.exp(-2j * math.pi * np.outer(fs, t)) @ y)
    f_scan = fs[np.argmax(mag)]
    assert abs(f_est - f_scan) < 1e-6


def test_strouhal_uses_the_final_quarter_and_scales():
    t = np.arange(40000)
    # a different frequency in the first three quarters must not count
    sig = np.where(t < 30000, np.sin(2 * math.pi * 0.005 * t), np.sin(2 * math.pi * 0.002 * t))
    assert abs(ost.strouhal(sig, L=20, u_inf=0.05) - 20 * 0.002 / 0.05) < 2e-4
