"""Trajectory error measures -- TEST INFRASTRUCTURE ONLY.

Great-circle distance between two positions on a sphere of radius R (haversine
form), used to report the error of reduced-precision and learned-surrogate
trajectories against plain float64 trajectories in kilometres.
"""
from __future__ import annotations

import numpy as np

R_EARTH = 6371000.0


def great_circle_km(lon1, lat1, lon2, lat2):
    l1, p1, l2, p2 = (np.radians(np.asarray(a, dtype=np.float64)) for a in (lon1, lat1, lon2, lat2))
    h = np.sin((p2 - p1) / 2) ** 2 + np.cos(p1) * np.cos(p2) * np.sin((l2 - l1) / 2) ** 2
    return 2.0 * R_EARTH * np.arcsin(np.sqrt(np.clip(h, 0.0, 1.0))) / 1000.0


def lon_diff(a, b):
    """Signed longitude difference a - b folded into [-180, 180)."""
    return np.mod(np.asarray(a, float) - np.asarray(b, float) + 180.0, 360.0) - 180.0
