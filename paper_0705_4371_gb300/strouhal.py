"""Host-side Strouhal number estimator (Sec. 4.2.1).

The shedding frequency is the dominant frequency of the probe's u_x signal
over the final 25 % of the run.  The paper names the discrete Fourier
transform; a plain periodogram's bin width over a few thousand samples is
several per cent of St, so this estimator removes the mean, applies a Hann
window, zero-pads by 8 and refines the peak bin by parabolic interpolation
of the log-magnitude.  The same function is applied to the GPU's and the
oracle's probe signals.
"""
import numpy as np


def dominant_frequency(signal, dt=1.0, tail=0.25, pad=8):
    x = np.asarray(signal, np.float64)
    x = x[int(round(len(x) * (1.0 - tail))):]
    if x.size < 8:
        raise ValueError("signal too short for a frequency estimate")
    x = (x - x.mean()) * np.hanning(x.size)
    n = int(2 ** np.ceil(np.log2(x.size * pad)))
    mag = np.abs(np.fft.rfft(x, n))
    k = int(np.argmax(mag[1:]) + 1)
    if 1 <= k < mag.size - 1:
        a, b, c = np.log(mag[k - 1] + 1e-300), np.log(mag[k] + 1e-300), np.log(mag[k + 1] + 1e-300)
        den = a - 2 * b + c
        off = 0.5 * (a - c) / den if den != 0 else 0.0
    else:
        off = 0.0
    return (k + off) / (n * dt)


def strouhal(signal, L, u_inf, dt=1.0, tail=0.25):
    """St = L f / u_inf with f the dominant frequency of the signal tail."""
    return L * dominant_frequency(signal, dt, tail) / u_inf
