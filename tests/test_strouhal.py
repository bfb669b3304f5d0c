"""The host-side Strouhal estimator recovers a known frequency (Sec. 4.2.1)."""
import math

import numpy as np

from paper_0705_4371_gb300 import inputs, strouhal


def test_recovers_sinusoid_frequency():
    for f0 in (0.00137, 0.0021, 0.0113):
        t = np.arange(40000)
        noise = inputs.uniform(7, (t.size,), -0.2, 0.2)
        sig = 0.05 + 0.01 * np.sin(2 * math.pi * f0 * t + 0.3) + 0.001 * noise
        f = strouhal.dominant_frequency(sig)
        assert abs(f / f0 - 1) < 1e-4


def test_strouhal_scaling():
    t = np.arange(20000)
    sig = np.sin(2 * math.pi * 0.002 * t)
    assert abs(strouhal.strouhal(sig, L=20, u_inf=0.05) - 20 * 0.002 / 0.05) < 1e-4
