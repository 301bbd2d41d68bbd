"""Physical constants of the oracle (SI).  Time convention e^{i omega t} (Sec. IV-B)."""
import math

C0 = 299792458.0            # speed of light in vacuum, m/s
MU0 = 4.0e-7 * math.pi      # vacuum permeability, H/m


def k0(freq_hz: float) -> float:
    """Free-space wavenumber omega / c0."""
    return 2.0 * math.pi * freq_hz / C0


def omega(freq_hz: float) -> float:
    return 2.0 * math.pi * freq_hz
