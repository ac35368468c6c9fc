"""Windowed harmonic spectrum and per-harmonic yields.

TEST INFRASTRUCTURE (oracle). Paper Sec. "Dipoles": S(w) = |int a(t) W(t) e^{iwt} dt|^2
~ w^4 |int d(t) W(t) e^{iwt} dt|^2 with an apodisation W(t) such as a Kaiser window.
Readings: Kaiser beta = 8 over the whole record, FFT zero-padded to a power of two
>= 8x the record length; yield of odd harmonic q = integral of S over
[(q - 1/2) w0, (q + 1/2) w0] (trapezoid rule); cutoff I_p + 3.17 U_p (Sec. Molecular HHG)
with U_p = E0^2 / (4 m w0^2).
"""
from __future__ import annotations

import numpy as np


def spectrum(signal, dt, beta=8.0, pad_factor=8, length_form=False):
    sig = np.asarray(signal, dtype=np.float64)
    n = sig.shape[0]
    w = np.kaiser(n, beta)
    N = 1
    while N < pad_factor * n:
        N *= 2
    F = np.fft.rfft(sig * w, N) * dt
    omega = 2.0 * np.pi * np.arange(F.shape[0]) / (N * dt)
    S = np.abs(F) ** 2
    if length_form:
        S = S * omega ** 4
    return omega, S


def harmonic_yields(omega, S, omega0, qmax):
    qs = np.arange(1, int(qmax) + 1, 2)
    out = []
    for q in qs:
        sel = (omega >= (q - 0.5) * omega0) & (omega <= (q + 0.5) * omega0)
        out.append(np.trapezoid(S[sel], omega[sel]) if np.count_nonzero(sel) > 1 else 0.0)
    return qs, np.asarray(out)


def cutoff_harmonic(ip, e0, omega0, m_eff=1.0):
    up = e0 * e0 / (4.0 * m_eff * omega0 * omega0)
    return (ip + 3.17 * up) / omega0
