"""Measurement grid and sputter-rate calibration data (inputs only).

* 342 measurement areas per 100 mm library (Sec. "Setup of the sputter
  system": EDS on 342 areas).  Their coordinates are not published, so the
  stand-in is a square grid of pitch 4 mm clipped to a 90 mm diameter, keeping
  the 342 points nearest the centre; each point is the 8 x 8 block of 0.5 mm
  tally cells around it (a 4 mm square patch).
* Sputter-rate calibration points from Table S1 (deposition time, average
  thickness, power) for the power-supply pairing each cathode uses in Table 1
  (Ni DC, Pd RF, Pt DC, Ru DC).  The "27 60" of the garbled Ni 35 W row is
  read as 2760 s (101.7 nm / 2760 s = 0.03685 nm/s, the printed rate).
* Power ranges of Table 1 (W) and the bulk densities of elements.py are used
  to draw synthetic target libraries.
"""

from __future__ import annotations

import numpy as np

# element -> list of (power W, deposition time s, average thickness nm, printed rate nm/s), Table S1
TABLE_S1 = {
    "Ni": {"DC": [(5.0, 28800.0, 165.5, 0.005745), (35.0, 2760.0, 101.7, 0.03685)],
           "RF": [(7.0, 28800.0, 95.7, 0.003323), (30.0, 7200.0, 99.3, 0.0138)]},
    "Pd": {"DC": [(5.0, 5400.0, 133.4, 0.0247), (30.0, 1200.0, 178.0, 0.1483)],
           "RF": [(7.0, 14400.0, 70.0, 0.004861), (60.0, 1080.0, 83.5, 0.07731)]},
    "Pt": {"DC": [(5.0, 9960.0, 140.5, 0.01411), (35.0, 960.0, 102.4, 0.1067)]},
    "Ru": {"DC": [(5.0, 18000.0, 97.6, 0.005422), (35.0, 1800.0, 90.5, 0.05028)]},
}
# element -> supply -> [(power W, discharge voltage V)], the voltage column of Table S1
VOLTAGE_S1 = {
    "Ni": {"DC": [(5.0, 289.0), (35.0, 294.0)], "RF": [(7.0, 25.0), (30.0, 33.0)]},
    "Pd": {"DC": [(5.0, 294.0), (30.0, 299.0)], "RF": [(7.0, 29.0), (60.0, 49.0)]},
    "Pt": {"DC": [(5.0, 306.0), (35.0, 323.0)]},
    "Ru": {"DC": [(5.0, 262.0), (35.0, 272.0)]},
}
# supply pairing of Table 1 (all libraries but the equiatomic one)
SUPPLY = {"Ni": "DC", "Pd": "RF", "Pt": "DC", "Ru": "DC"}
# power set-points of Table 1 per element (W), the range the synthetic targets are drawn from
POWER_RANGE = {"Ni": (5.0, 35.0), "Pd": (7.0, 60.0), "Pt": (5.0, 35.0), "Ru": (5.0, 35.0)}


def calibration_points(symbol: str):
    """The two (power W, rate nm/s) points of Table S1 for the element's supply,
    with the rate taken as thickness / time."""
    rows = TABLE_S1[symbol][SUPPLY[symbol]]
    return [(p, thick / t) for (p, t, thick, _printed) in rows]


def measurement_patches(nx=200, ny=200, half_u=50.0, half_v=50.0, pitch=4.0, diameter=90.0, n_points=342):
    """Patch id of every tally cell (-1 outside every patch), point coordinates
    (u, v) in mm, and the index of the central (reference) point."""
    du, dv = 2 * half_u / nx, 2 * half_v / ny
    k = int(diameter / 2 // pitch) + 1
    pts = [(i * pitch, j * pitch) for i in range(-k, k + 1) for j in range(-k, k + 1)
           if (i * pitch) ** 2 + (j * pitch) ** 2 <= (diameter / 2) ** 2]
    pts.sort(key=lambda q: (q[0] ** 2 + q[1] ** 2, q[0], q[1]))
    pts = np.array(pts[:n_points], dtype=np.float64)
    patch = -np.ones(nx * ny, dtype=np.int32)
    uc = -half_u + du * (np.arange(nx) + 0.5)
    vc = -half_v + dv * (np.arange(ny) + 0.5)
    for m, (u, v) in enumerate(pts):
        ix = np.nonzero(np.abs(uc - u) < pitch / 2)[0]
        iy = np.nonzero(np.abs(vc - v) < pitch / 2)[0]
        for y in iy:
            patch[y * nx + ix] = m
    ref = int(np.argmin(pts[:, 0] ** 2 + pts[:, 1] ** 2))
    return patch, pts, ref


def voltage_points(symbol: str):
    """The two (power W, voltage V) points of Table S1 for the element's supply
    (DC: discharge voltage; RF: bias)."""
    return list(VOLTAGE_S1[symbol][SUPPLY[symbol]])
