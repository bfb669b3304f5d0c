"""Strouhal number of a probe signal, oracle side (test infrastructure only).

Sec. 4.2.1 takes the shedding frequency as the dominant frequency of the
probe's u_x signal and St = L f / u_inf.  The paper names the discrete
Fourier transform; the estimator of this reading: the final quarter of the
signal, its mean removed, a Hann window w_n = 1/2 - 1/2 cos(2 pi n / (N - 1)),
the DFT zero-padded to 8 N points, and the peak refined by the parabola
through the logarithms of the peak bin and its two neighbours.  Written for
the oracle on its own (numpy's FFT as the DFT primitive); pinned by CPU
tests against known sinusoids and a direct scan of the windowed DFT.
"""
import numpy as np


def peak_frequency(x, pad=8):
    """Frequency (cycles per sample) of the largest windowed-DFT peak of x."""
    x = np.asarray(x, np.float64)
    n = x.size
    w = 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(n) / (n - 1))
    y = (x - x.mean()) * w
    m = pad * n
    a = np.abs(np.fft.rfft(y, m))
    k = 1 + int(np.argmax(a[1:]))
    if k + 1 >= a.size:
        return k / m
    l0, l1, l2 = np.log(a[k - 1]), np.log(a[k]), np.log(a[k + 1])
    curv = l0 - 2.0 * l1 + l2
    shift = 0.0 if curv == 0.0 else 0.5 * (l0 - l2) / curv
    return (k + shift) / m


def strouhal(probe_ux, L, u_inf, tail=0.25):
    """St = L f / u_inf from the final `tail` fraction of the probe signal."""
    x = np.asarray(probe_ux, np.float64)
    x = x[len(x) - int(round(len(x) * tail)):]
    return L * peak_frequency(x) / u_inf
