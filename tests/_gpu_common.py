"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest
import torch

from oracle.errors import great_circle_km, lon_diff

KM_PER_DEG = 6371.0 * np.pi / 180.0

# Tolerances of the FP32 kernels against the FP64 oracle after 120 steps:
# 1e-4 degrees in longitude/latitude and 1e-5 relative in pressure.
TOL_DEG = 1e-4
TOL_P = 1e-5


@pytest.fixture(scope="session")
def M():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2211_12616_gb300 as mod
    mod.load()
    return mod


def make_ctx(M, grid, snaps, times, storage=0, nvars=3, device=True):
    ctx = M.Context(grid, storage, nvars)
    for slot, (s, t) in enumerate(zip(snaps, times)):
        if device:
            d = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in s.items()}
            ctx.load_met(slot, t, d["u"], d["v"], d["w"], d.get("T"))
        else:
            ctx.load_met(slot, t, s["u"], s["v"], s["w"], s.get("T"))
    torch.cuda.synchronize()
    return ctx


def by_id(d):
    order = np.argsort(d["id"], kind="stable")
    return {k: np.asarray(v)[order] for k, v in d.items()}


def assert_positions_close(got, ref, tol_deg=TOL_DEG, tol_p=TOL_P, what="", lon_metric="deg"):
    """Positions agree within tol_deg (degrees) and tol_p (relative pressure).

    lon_metric "deg": |dlon| (folded into [-180, 180)) <= tol_deg, the literal
    criterion, used for deterministic advection.  "arc": the great-circle
    distance in degrees of arc <= tol_deg -- for stochastic runs, where within
    a fraction of a degree of a pole a sub-millimetre displacement difference
    is already 1e-4 degrees of longitude.  |dlat| <= tol_deg in both cases.
    """
    dlon = np.abs(lon_diff(got["lon"], ref["lon"]))
    arc = great_circle_km(got["lon"], got["lat"], ref["lon"], ref["lat"]) / KM_PER_DEG
    dlat = np.abs(got["lat"] - ref["lat"])
    dp = np.abs(got["p"] - ref["p"]) / ref["p"]
    msg = (f"{what}: max |dlon| {dlon.max():.3e} deg, max arc {arc.max():.3e} deg, "
           f"max |dlat| {dlat.max():.3e} deg, max |dp|/p {dp.max():.3e}")
    horiz = dlon.max() if lon_metric == "deg" else arc.max()
    assert horiz <= tol_deg and dlat.max() <= tol_deg and dp.max() <= tol_p, msg
    return dlon.max(), dlat.max(), dp.max()
