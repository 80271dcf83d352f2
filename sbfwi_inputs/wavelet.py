"""Source time functions, sampled on the host so that every consumer gets identical samples."""

import numpy as np


def ricker(f0: float, dt: float, K: int, t0: float | None = None, amplitude: float = 1.0) -> np.ndarray:
    """Ricker wavelet r(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2).

    Sampled at t_k = k*dt for k = 1..K (the sample that drives the Newmark step that
    produces the state at t_k).  The default delay t0 = 1.5/f0 makes r(0) about
    1e-8 of the peak, so zero initial conditions are consistent.
    """
    if t0 is None:
        t0 = 1.5 / f0
    t = np.arange(1, K + 1, dtype=np.float64) * dt
    a = (np.pi * f0 * (t - t0)) ** 2
    return amplitude * (1.0 - 2.0 * a) * np.exp(-a)


def sine_burst(f0: float, dt: float, K: int, cycles: int = 2, amplitude: float = 1.0) -> np.ndarray:
    """Tone burst a sin(2 pi f0 t) sin^2(pi f0 t / cycles) for 0 <= t <= cycles/f0, zero after
    (a sine carrier under a sin^2 window of `cycles` carrier periods), sampled at
    t_k = k*dt for k = 1..K like ``ricker``."""
    t = np.arange(1, K + 1, dtype=np.float64) * dt
    w = np.where(t <= cycles / f0, np.sin(np.pi * f0 * t / cycles) ** 2, 0.0)
    return amplitude * np.sin(2.0 * np.pi * f0 * t) * w
